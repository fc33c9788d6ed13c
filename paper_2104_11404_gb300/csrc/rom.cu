// Hyper-reduced online step of the reduced order model (Section 3): the
// RK2-average scheme in reduced coordinates (eq:RK2-avg-rom-hr) with the SNS
// nonlinear-term bases of Section 4.2 (eq:rom-hr-sns) and DEIM sampling
// (Section 4.3), under the step control of Section 2.2.3.
//
// Set-up (lh_rom_create, host and device, once): the SNS bases Phi_F =
// M_V Phi_v (essential rows zero, as those of F.1) and Phi_G = M_E Phi_e; the
// DEIM rows Z_F, Z_G (greedy, with over-sampling) unless the caller gives
// them; the least-squares matrices A_F = (Z_F^T Phi_F)^+ and A_G =
// (Z_G^T Phi_G)^+ (Householder QR); the sampled elements (every element
// touching a sampled F.1 node, the element of every sampled F^T w entry); the
// basis rows at the nodes and energy dofs of those elements; the tables that
// gather a sampled entry from the element rows of the restricted force; and
// C = Phi_x^T Phi_v, b = Phi_x^T v_os for the position equation.
//
// Online step (one CUDA graph per attempt, every scalar on the device; one
// restricted force evaluation per stage):
//   stage s = 0, 1:
//     lift the stage coordinates at the sampled rows (eq:discretesolrepresentation)
//     restricted force on the sampled elements -> F.1 at Z_F, estimate
//     f = A_F Z_F^T F.1 and the velocity update (single CTA)
//     lift the test velocity (v^{n+1/2}, then the average) at the sampled rows
//     F^T w of the sampled elements from the stress weights the force kept -> F^T w at Z_G
//     g = A_G Z_G^T F^T w and the energy and position updates (single CTA)
//   control (Section 2.2.3) and commit.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <set>
#include <vector>

#include "control.cuh"

struct lh_rom {
  lh_ctx* ctx = nullptr;
  int nbv = 0, nbe = 0, nbx = 0;  // basis sizes
  int nsf = 0, nsg = 0;           // sampled F.1 / F^T w entries
  int64_t nsel = 0;               // sampled elements
  int64_t nrv = 0, nre = 0;       // lifted rows (kinematic, thermodynamic)
  std::vector<int64_t> hsf, hsg;  // sample rows
  std::vector<int32_t> hsel;      // sampled elements
  // device
  int32_t* sel = nullptr;
  int64_t* rows_v = nullptr;      // kinematic rows lifted (c * nnodes + node)
  int64_t* rows_e = nullptr;      // thermodynamic rows lifted
  double *Pv = nullptr, *Px = nullptr, *Pe = nullptr;  // basis rows [row][basis]
  double *vos = nullptr, *xos = nullptr, *eos = nullptr;  // offsets at those rows
  double *AF = nullptr, *AG = nullptr;  // [basis][sample]
  int32_t *gf_off = nullptr, *gf_idx = nullptr;  // F.1 sample s: flat element-row indices
  int32_t* gg_idx = nullptr;                     // F^T w sample s: flat index
  double *C = nullptr, *bx = nullptr;  // Phi_x^T Phi_v [nbx][nbv], Phi_x^T v_os
  // full-size bases and offsets (kept for lh_rom_lift)
  double *Phv = nullptr, *Phe = nullptr, *Phx = nullptr, *fvos = nullptr, *feos = nullptr,
         *fxos = nullptr;
  // reduced state (device): current, half step, candidate, average
  double* red = nullptr;          // 3 x (nbv + nbe + nbx) + nbv + nbv + nbe
  double *vh, *eh, *xh, *vh2, *eh2, *xh2, *vhn, *ehn, *xhn, *vbar, *fh, *gh;
  double *vF = nullptr, *eF = nullptr, *xF = nullptr, *wF = nullptr;  // lifting buffers
  double *F1E = nullptr, *FTvE = nullptr;
  lagh::Ctl* ctl = nullptr;
  lagh::Ctl* ctl_host = nullptr;
  cudaGraphExec_t graph = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  std::string err;
};

namespace lagh {

static lh_status rom_error(lh_rom* r, lh_status s, const char* msg) {
  if (r) r->err = msg;
  return s;
}

static lh_status rom_cuda(lh_rom* r, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return LH_OK;
  char buf[256];
  snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
  if (r) r->err = buf;
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? LH_ENOMEM : LH_ECUDA;
}

// out[rows[i]] = os[i] + sum_j P[i][j] c[j] for the nr listed rows.
__global__ void rom_lift_kernel(int64_t nr, int nb, const double* __restrict__ P,
                                const double* __restrict__ os, const int64_t* __restrict__ rows,
                                const double* __restrict__ c, double* __restrict__ out,
                                const Ctl* ctl) {
  pdl_enter();
  if (ctl != nullptr && ctl->done) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nr;
       i += (int64_t)gridDim.x * blockDim.x) {
    double s = os[i];
    const double* p = P + i * nb;
    for (int j = 0; j < nb; ++j) s = fma(p[j], c[j], s);
    out[rows[i]] = s;
  }
}

// The three lifts of a stage state in one launch: rows [0, nrv) of v,
// [nrv, nrv + nre) of e, [nrv + nre, 2 nrv + nre) of x (x uses v's rows);
// each row as rom_lift_kernel forms it.
__global__ void rom_lift3_kernel(int64_t nrv, int64_t nre, int nbv, int nbe, int nbx,
                                 const double* __restrict__ Pv, const double* __restrict__ vos,
                                 const int64_t* __restrict__ rows_v, const double* __restrict__ cv,
                                 double* __restrict__ vF, const double* __restrict__ Pe,
                                 const double* __restrict__ eos, const int64_t* __restrict__ rows_e,
                                 const double* __restrict__ ce, double* __restrict__ eF,
                                 const double* __restrict__ Px, const double* __restrict__ xos,
                                 const double* __restrict__ cx, double* __restrict__ xF,
                                 const Ctl* ctl) {
  pdl_enter();
  if (ctl != nullptr && ctl->done) return;
  const int64_t n = 2 * nrv + nre;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const double *P, *os, *c;
    const int64_t* rows;
    double* out;
    int nb;
    int64_t i;
    if (t < nrv) { i = t; P = Pv; os = vos; rows = rows_v; c = cv; out = vF; nb = nbv; }
    else if (t < nrv + nre) { i = t - nrv; P = Pe; os = eos; rows = rows_e; c = ce; out = eF; nb = nbe; }
    else { i = t - nrv - nre; P = Px; os = xos; rows = rows_v; c = cx; out = xF; nb = nbx; }
    double s = os[i];
    const double* p = P + i * nb;
    for (int j = 0; j < nb; ++j) s = fma(p[j], c[j], s);
    out[rows[i]] = s;
  }
}

struct RomStage {
  int stage;   // 0 or 1
  int which;   // 0: F.1 part (velocity), 1: F^T w part (energy, position)
};

// Projection of the sampled entries and the reduced update of one part of a
// stage, one CTA (the reduced sizes are small).  Each matrix-vector product
// gives one row to one warp: the lanes take every 32nd column and the warp
// adds them by a fixed shuffle tree.
__device__ __forceinline__ double row_dot(const double* __restrict__ row, const double* x, int n,
                                          int lane) {
  double acc = 0.0;
  for (int s = lane; s < n; s += 32) acc = fma(row[s], x[s], acc);
  return warp_sum(acc);
}

__global__ void __launch_bounds__(1024) rom_update_kernel(
    RomStage rs, int nbv, int nbe, int nbx, int nsf, int nsg, const double* __restrict__ F1E,
    const double* __restrict__ FTvE, const int32_t* __restrict__ gf_off,
    const int32_t* __restrict__ gf_idx, const int32_t* __restrict__ gg_idx,
    const double* __restrict__ AF, const double* __restrict__ AG, const double* __restrict__ C,
    const double* __restrict__ bx, double* vh, double* eh, double* xh, double* vh2, double* eh2,
    double* xh2, double* vhn, double* ehn, double* xhn, double* vbar, double* fh, double* gh,
    const Ctl* ctl, Ctl* ctlw, CtlConsts k) {
  pdl_enter();
  if (ctl->done) return;
  extern __shared__ double zs[];
  const double dt = ctl->dt_use;
  const int tid = threadIdx.x;
  if (rs.which == 0) {
    // z = Z_F^T F.1: each sampled entry is the sum of its element rows, in
    // the table's (element) order
    for (int s = tid; s < nsf; s += blockDim.x) {
      double acc = 0.0;
      for (int q = gf_off[s]; q < gf_off[s + 1]; ++q) acc += F1E[gf_idx[q]];
      zs[s] = acc;
    }
    __syncthreads();
    for (int j = tid >> 5; j < nbv; j += blockDim.x >> 5) {
      const double acc = row_dot(AF + (int64_t)j * nsf, zs, nsf, tid & 31);
      if ((tid & 31) == 0) fh[j] = acc;
    }
    __syncthreads();
    for (int j = tid; j < nbv; j += blockDim.x) {
      if (rs.stage == 0) {
        vh2[j] = vh[j] - 0.5 * dt * fh[j];
      } else {
        const double v1 = vh[j] - dt * fh[j];
        vhn[j] = v1;
        vbar[j] = 0.5 * (vh[j] + v1);
      }
    }
  } else {
    for (int s = tid; s < nsg; s += blockDim.x) zs[s] = FTvE[gg_idx[s]];
    __syncthreads();
    for (int j = tid >> 5; j < nbe; j += blockDim.x >> 5) {
      const double acc = row_dot(AG + (int64_t)j * nsg, zs, nsg, tid & 31);
      if ((tid & 31) == 0) gh[j] = acc;
    }
    __syncthreads();
    const double* w = rs.stage == 0 ? vh2 : vbar;
    const double c = rs.stage == 0 ? 0.5 * dt : dt;
    for (int j = tid; j < nbe; j += blockDim.x) (rs.stage == 0 ? eh2 : ehn)[j] = eh[j] + c * gh[j];
    for (int j = tid >> 5; j < nbx; j += blockDim.x >> 5) {
      // Phi_x^T (v_os + Phi_v w) = bx + C w
      const double d = row_dot(C + (int64_t)j * nbv, w, nbv, tid & 31);
      if ((tid & 31) == 0) (rs.stage == 0 ? xh2 : xhn)[j] = xh[j] + c * (bx[j] + d);
    }
  }
  if (ctlw != nullptr) {
    // end of the attempt (ctlw = the control block): the step control, and
    // the commit of the candidate coordinates vhn, ehn, xhn (contiguous, as
    // are vh, eh, xh) if accepted
    __shared__ int acc;
    __syncthreads();
    if (tid == 0) {
      control_update(ctlw, k);
      acc = ctlw->accepted;
    }
    __syncthreads();
    if (acc)
      for (int j = tid; j < nbv + nbe + nbx; j += blockDim.x) vh[j] = vhn[j];
  }
}

__global__ void rom_begin_kernel(Ctl* ctl, double t_final, long long max_steps, double dt_min,
                                 int fixed, double dt_fixed, const unsigned long long* est) {
  if (threadIdx.x == 0 && blockIdx.x == 0)
    control_begin(ctl, t_final, max_steps, dt_min, fixed, dt_fixed, nullptr, 0, est);
}

// out = os + Phi c over all N rows (Phi column-major N x nb).
__global__ void rom_lift_full_kernel(int64_t N, int nb, const double* __restrict__ Phi,
                                     const double* __restrict__ os, const double* __restrict__ c,
                                     double* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    double s = os[i];
    for (int j = 0; j < nb; ++j) s = fma(Phi[(int64_t)j * N + i], c[j], s);
    out[i] = s;
  }
}

__global__ void rom_set_bits_kernel(unsigned long long* p, int* flag) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    *p = kInfBits;
    *flag = 0;
  }
}

// ------------------------------------------------------------ host set-up --

// Householder QR least squares: returns A^+ (n x m, row-major) of the m x n
// matrix B (row-major, m >= n, full column rank), or false if rank-deficient.
static bool pinv_qr(int m, int n, const std::vector<double>& B, std::vector<double>& Ap) {
  std::vector<double> R(B);                     // m x n, overwritten
  std::vector<double> Q((size_t)m * m, 0.0);    // accumulated orthogonal factor
  for (int i = 0; i < m; ++i) Q[(size_t)i * m + i] = 1.0;
  std::vector<double> u(m);
  for (int k = 0; k < n; ++k) {
    double nrm = 0.0;
    for (int i = k; i < m; ++i) nrm += R[(size_t)i * n + k] * R[(size_t)i * n + k];
    nrm = sqrt(nrm);
    if (nrm == 0.0) return false;
    const double alpha = R[(size_t)k * n + k] > 0 ? -nrm : nrm;
    for (int i = 0; i < m; ++i) u[i] = 0.0;
    u[k] = R[(size_t)k * n + k] - alpha;
    for (int i = k + 1; i < m; ++i) u[i] = R[(size_t)i * n + k];
    double un = 0.0;
    for (int i = k; i < m; ++i) un += u[i] * u[i];
    if (un == 0.0) continue;
    for (int j = k; j < n; ++j) {  // R <- (I - 2 u u^T / u^T u) R
      double s = 0.0;
      for (int i = k; i < m; ++i) s += u[i] * R[(size_t)i * n + j];
      s *= 2.0 / un;
      for (int i = k; i < m; ++i) R[(size_t)i * n + j] -= s * u[i];
    }
    for (int r = 0; r < m; ++r) {  // Q <- Q (I - 2 u u^T / u^T u)
      double s = 0.0;
      for (int i = k; i < m; ++i) s += Q[(size_t)r * m + i] * u[i];
      s *= 2.0 / un;
      for (int i = k; i < m; ++i) Q[(size_t)r * m + i] -= s * u[i];
    }
  }
  double rmax = 0.0;
  for (int k = 0; k < n; ++k) rmax = std::max(rmax, fabs(R[(size_t)k * n + k]));
  for (int k = 0; k < n; ++k)
    if (!(fabs(R[(size_t)k * n + k]) > 1e-13 * rmax)) return false;
  // A^+ = R1^{-1} Q1^T: solve R1 X = Q1^T column by column
  Ap.assign((size_t)n * m, 0.0);
  for (int col = 0; col < m; ++col) {
    for (int k = n - 1; k >= 0; --k) {
      double s = Q[(size_t)col * m + k];  // (Q^T)[k][col]
      for (int l = k + 1; l < n; ++l) s -= R[(size_t)k * n + l] * Ap[(size_t)l * m + col];
      Ap[(size_t)k * m + col] = s / R[(size_t)k * n + k];
    }
  }
  return true;
}

// Greedy DEIM with over-sampling: basis vector j receives its share of the ns
// rows, each at the largest entry of the residual of its least-squares
// reconstruction, from the rows chosen so far, by the basis vectors before it
// (ns = m: the classical greedy DEIM).  Phi: N x m column-major.  Ties go to
// the lowest row index.
static bool deim_select(int64_t N, int m, int ns, const std::vector<double>& Phi,
                        std::vector<int64_t>& p) {
  p.clear();
  std::vector<char> used(N, 0);
  std::vector<double> r(N), B, Ap;
  for (int j = 0; j < m; ++j) {
    const int share = ns / m + (j < ns % m ? 1 : 0);
    for (int t = 0; t < share; ++t) {
      if (j == 0) {
        for (int64_t i = 0; i < N; ++i) r[i] = Phi[i];
      } else {
        const int np = (int)p.size();
        if (np < j) return false;
        B.assign((size_t)np * j, 0.0);
        for (int a = 0; a < np; ++a)
          for (int l = 0; l < j; ++l) B[(size_t)a * j + l] = Phi[(size_t)l * N + p[a]];
        if (!pinv_qr(np, j, B, Ap)) return false;
        std::vector<double> c(j, 0.0);
        for (int l = 0; l < j; ++l)
          for (int a = 0; a < np; ++a) c[l] += Ap[(size_t)l * np + a] * Phi[(size_t)j * N + p[a]];
        for (int64_t i = 0; i < N; ++i) {
          double s = Phi[(size_t)j * N + i];
          for (int l = 0; l < j; ++l) s -= Phi[(size_t)l * N + i] * c[l];
          r[i] = s;
        }
      }
      int64_t best = -1;
      double bv = -1.0;
      for (int64_t i = 0; i < N; ++i)
        if (!used[i] && fabs(r[i]) > bv) { bv = fabs(r[i]); best = i; }
      if (best < 0) return false;
      used[best] = 1;
      p.push_back(best);
    }
  }
  return true;
}

template <typename T>
static cudaError_t up(T** d, const std::vector<T>& h) {
  cudaError_t e = cudaMalloc((void**)d, std::max<size_t>(h.size(), 1) * sizeof(T));
  if (e == cudaSuccess && !h.empty())
    e = cudaMemcpy(*d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
  return e;
}

static void rom_free(lh_rom* r) {
  void* ptrs[] = {r->sel, r->rows_v, r->rows_e, r->Pv, r->Px, r->Pe, r->vos, r->xos, r->eos,
                  r->AF, r->AG, r->gf_off, r->gf_idx, r->gg_idx, r->C, r->bx, r->Phv, r->Phe,
                  r->Phx, r->fvos, r->feos, r->fxos, r->red, r->vF, r->eF, r->xF, r->wF, r->F1E,
                  r->FTvE, r->ctl};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (r->ctl_host) cudaFreeHost(r->ctl_host);
  if (r->graph) cudaGraphExecDestroy(r->graph);
  if (r->ev0) cudaEventDestroy(r->ev0);
  if (r->ev1) cudaEventDestroy(r->ev1);
}

static int node_of(const Geom& g, const int* I) {
  return I[0] + g.nn[0] * (I[1] + (g.dim == 3 ? g.nn[1] * I[2] : 0));
}

// Global nodes of element el.
static void element_nodes(const Geom& g, int64_t el, std::vector<int64_t>& out) {
  const int k = g.k, P = k + 1;
  int E[3] = {(int)(el % g.n[0]), (int)((el / g.n[0]) % g.n[1]),
              (int)(el / ((int64_t)g.n[0] * g.n[1]))};
  const int nd1 = g.dim == 3 ? P * P * P : P * P;
  out.resize(nd1);
  for (int i = 0; i < nd1; ++i) {
    int I[3] = {E[0] * k + i % P, E[1] * k + (i / P) % P, g.dim == 3 ? E[2] * k + i / (P * P) : 0};
    out[i] = node_of(g, I);
  }
}

// ------------------------------------------------------------- the step --

static cudaError_t rom_enqueue_attempt(lh_rom* r, cudaStream_t s) {
  lh_ctx* c = r->ctx;
  const Geom& g = c->g;
  const bool pdl = c->use_pdl != 0;
  const int lb = 256;
  auto blocks = [&](int64_t n) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + lb - 1) / lb, 1024)); };
  const int nd1 = g.dim == 3 ? (g.k + 1) * (g.k + 1) * (g.k + 1) : (g.k + 1) * (g.k + 1);
  (void)nd1;
  const size_t zsm = sizeof(double) * (size_t)std::max(r->nsf, r->nsg);
  const bool mixed = c->precision == LH_MIXED;
  CtlConsts k;
  k.beta1 = c->phys_desc.beta1;
  k.beta2 = c->phys_desc.beta2;
  k.gamma_dt = c->phys_desc.gamma_dt;
  cudaError_t e;
  for (int st = 0; st < 2; ++st) {
    const double* cv = st == 0 ? r->vh : r->vh2;
    const double* ce = st == 0 ? r->eh : r->eh2;
    const double* cx = st == 0 ? r->xh : r->xh2;
    // lift the stage state at the sampled rows (v, e, x in one launch)
    if ((e = launch_k(pdl, rom_lift3_kernel, dim3(blocks(2 * r->nrv + r->nre)), dim3(lb), 0, s,
                      r->nrv, r->nre, r->nbv, r->nbe, r->nbx, (const double*)r->Pv,
                      (const double*)r->vos, (const int64_t*)r->rows_v, cv, r->vF,
                      (const double*)r->Pe, (const double*)r->eos, (const int64_t*)r->rows_e, ce,
                      r->eF, (const double*)r->Px, (const double*)r->xos, cx, r->xF,
                      (const Ctl*)r->ctl)) != cudaSuccess)
      return e;
    // restricted force: F.1 element rows and the estimate of this stage
    ForceArgs f = {};
    f.v = r->vF; f.e = r->eF; f.x = r->xF; f.vtest = nullptr;
    f.list = r->sel; f.nslots = r->nsel;
    f.F1E = r->F1E;
    // kept for F^T w below: the stress weights (FP64) or the FP32 element
    // matrices (mixed) of the sampled elements
    f.D = mixed ? nullptr : c->a.D;
    f.FK = mixed ? c->a.FK : nullptr;
    f.tau_bits = &r->ctl->tau_bits[st];
    f.status = &r->ctl->status;
    f.ctl = r->ctl;
    f.p_ref = &c->a.ctl->p_ref;
    f.mode = kForceFull;
    if ((e = launch_force(c, f, s)) != cudaSuccess) return e;
    RomStage rs = {st, 0};
    if ((e = launch_k(pdl, rom_update_kernel, dim3(1), dim3(1024), zsm, s, rs, r->nbv, r->nbe, r->nbx,
                      r->nsf, r->nsg, (const double*)r->F1E, (const double*)r->FTvE,
                      (const int32_t*)r->gf_off, (const int32_t*)r->gf_idx,
                      (const int32_t*)r->gg_idx, (const double*)r->AF, (const double*)r->AG,
                      (const double*)r->C, (const double*)r->bx, r->vh, r->eh, r->xh, r->vh2,
                      r->eh2, r->xh2, r->vhn, r->ehn, r->xhn, r->vbar, r->fh, r->gh,
                      (const Ctl*)r->ctl, (Ctl*)nullptr, k)) != cudaSuccess)
      return e;
    // the test velocity of the energy equation, lifted at the sampled rows
    const double* cw = st == 0 ? r->vh2 : r->vbar;
    if ((e = launch_k(pdl, rom_lift_kernel, dim3(blocks(r->nrv)), dim3(lb), 0, s, r->nrv, r->nbv,
                      (const double*)r->Pv, (const double*)r->vos, (const int64_t*)r->rows_v, cw,
                      r->wF, (const Ctl*)r->ctl)) != cudaSuccess)
      return e;
    // F^T w of the same force (the stress weights the force kernel kept)
    EnergyArgs ea = {};
    ea.w = r->wF;
    ea.D = c->a.D;
    ea.FK = c->a.FK;
    // mixed: the reference pressure's F^T w in FP64 from the stage positions
    ea.x = mixed ? r->xF : nullptr;
    ea.p_ref = mixed ? &c->a.ctl->p_ref : nullptr;
    ea.list = r->sel;
    ea.nslots = r->nsel;
    ea.FTvE = r->FTvE;
    ea.ctl = r->ctl;
    if ((e = launch_ftv_list(c, ea, s)) != cudaSuccess) return e;
    rs.which = 1;
    // the second stage's energy and position update also ends the attempt:
    // step control and commit in the same single-CTA kernel
    if ((e = launch_k(pdl, rom_update_kernel, dim3(1), dim3(1024), zsm, s, rs, r->nbv, r->nbe, r->nbx,
                      r->nsf, r->nsg, (const double*)r->F1E, (const double*)r->FTvE,
                      (const int32_t*)r->gf_off, (const int32_t*)r->gf_idx,
                      (const int32_t*)r->gg_idx, (const double*)r->AF, (const double*)r->AG,
                      (const double*)r->C, (const double*)r->bx, r->vh, r->eh, r->xh, r->vh2,
                      r->eh2, r->xh2, r->vhn, r->ehn, r->xhn, r->vbar, r->fh, r->gh,
                      (const Ctl*)r->ctl, st == 1 ? r->ctl : (Ctl*)nullptr, k)) != cudaSuccess)
      return e;
  }
  return cudaSuccess;
}

static lh_status rom_build_graph(lh_rom* r) {
  if (r->graph) return LH_OK;
  cudaStream_t s = r->ctx->work;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaError_t e2 = rom_enqueue_attempt(r, s);
    e = cudaStreamEndCapture(s, &g);
    if (e2 != cudaSuccess) e = e2;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&r->graph, g, 0);
  if (g) cudaGraphDestroy(g);
  if (e != cudaSuccess) r->graph = nullptr;
  return rom_cuda(r, e, "attempt graph");
}

static lh_status rom_read_ctl(lh_rom* r) {
  cudaStream_t s = r->ctx->work;
  cudaError_t e = cudaMemcpyAsync(r->ctl_host, r->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return rom_cuda(r, e, "read control block");
}

static lh_status rom_status(lh_rom* r) {
  const int st = r->ctl_host->status;
  if (st & kDevNonFinite) return rom_error(r, LH_ENONFINITE, "non-finite value in the lifted state");
  if (st & kDevDtMin) return rom_error(r, LH_EDTMIN, "time step collapsed below dt_min");
  return LH_OK;
}

// The estimate of the lifted current state over the sampled elements, into
// the context's scratch (ordered bits).
static cudaError_t rom_estimate(lh_rom* r, cudaStream_t s) {
  lh_ctx* c = r->ctx;
  unsigned long long* bits = reinterpret_cast<unsigned long long*>(c->a.aux + 8);
  int* flag = reinterpret_cast<int*>(c->a.aux + 9);
  rom_set_bits_kernel<<<1, 32, 0, s>>>(bits, flag);
  const int lb = 256;
  auto blocks = [&](int64_t n) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + lb - 1) / lb, 1024)); };
  rom_lift_kernel<<<blocks(r->nrv), lb, 0, s>>>(r->nrv, r->nbv, r->Pv, r->vos, r->rows_v, r->vh, r->vF, nullptr);
  rom_lift_kernel<<<blocks(r->nre), lb, 0, s>>>(r->nre, r->nbe, r->Pe, r->eos, r->rows_e, r->eh, r->eF, nullptr);
  rom_lift_kernel<<<blocks(r->nrv), lb, 0, s>>>(r->nrv, r->nbx, r->Px, r->xos, r->rows_v, r->xh, r->xF, nullptr);
  ForceArgs f = {};
  f.v = r->vF; f.e = r->eF; f.x = r->xF;
  f.list = r->sel; f.nslots = r->nsel;
  f.F1E = r->F1E;
  f.tau_bits = bits;
  f.status = flag;
  f.p_ref = &c->a.ctl->p_ref;
  f.mode = kForceFull;
  return launch_force(c, f, s);
}

static lh_status rom_run(lh_rom* r, double t_final, int64_t max_steps, int fixed, double dt_fixed,
                         float* wall_ms) {
  lh_ctx* c = r->ctx;
  cudaStream_t s = c->work;
  lh_status st;
  if ((st = rom_build_graph(r)) != LH_OK) return st;
  if (c->work != c->stream) {
    cudaEventRecord(r->ev0, c->stream);
    cudaStreamWaitEvent(s, r->ev0, 0);
  }
  if ((st = rom_read_ctl(r)) != LH_OK) return st;
  if (!fixed && !(r->ctl_host->dt > 0.0))
    if ((st = rom_cuda(r, rom_estimate(r, s), "estimate")) != LH_OK) return st;
  rom_begin_kernel<<<1, 32, 0, s>>>(r->ctl, t_final, (long long)max_steps,
                                   c->phys_desc.dt_min_frac * t_final, fixed, dt_fixed,
                                   reinterpret_cast<const unsigned long long*>(c->a.aux + 8));
  if ((st = rom_cuda(r, cudaGetLastError(), "begin")) != LH_OK) return st;
  if ((st = rom_read_ctl(r)) != LH_OK) return st;
  cudaEventRecord(r->ev0, s);
  const int64_t max_att = fixed ? 1 : INT64_MAX;
  int64_t att = 0;
  while (!r->ctl_host->done && att < max_att) {
    int64_t batch = 1;
    const Ctl& h = *r->ctl_host;
    if (!fixed && h.dt > 0.0) {
      const double rem = (h.t_final - h.t) / h.dt;
      batch = rem > 64.0 ? 64 : (int64_t)rem + 1;
      const int64_t left = h.max_steps - h.steps + 2;
      if (left < batch) batch = left > 1 ? left : 1;
    }
    for (int64_t i = 0; i < batch; ++i)
      if ((st = rom_cuda(r, cudaGraphLaunch(r->graph, s), "attempt launch")) != LH_OK) return st;
    att += batch;
    if ((st = rom_read_ctl(r)) != LH_OK) return st;
  }
  cudaEventRecord(r->ev1, s);
  if ((st = rom_cuda(r, cudaEventSynchronize(r->ev1), "run sync")) != LH_OK) return st;
  if (wall_ms) cudaEventElapsedTime(wall_ms, r->ev0, r->ev1);
  if (c->work != c->stream) {
    cudaEventRecord(r->ev1, s);
    cudaStreamWaitEvent(c->stream, r->ev1, 0);
  }
  return rom_status(r);
}

}  // namespace lagh

using namespace lagh;

extern "C" lh_status lh_rom_create(lh_ctx* c, const double* Phi_v, int32_t nbv, const double* Phi_e,
                                   int32_t nbe, const double* Phi_x, int32_t nbx, const double* v_os,
                                   const double* e_os, const double* x_os, int32_t nsf,
                                   int32_t nsg, const int64_t* samples_f,
                                   const int64_t* samples_g, lh_rom** out) {
  if (!out) return LH_EINVAL;
  *out = nullptr;
  if (!c || !Phi_v || !Phi_e || !Phi_x || !v_os || !e_os || !x_os) return LH_EINVAL;
  if (nbv < 1 || nbe < 1 || nbx < 1 || nbv > 1024 || nbe > 1024 || nbx > 1024) return LH_EINVAL;
  if (nsf < nbv || nsg < nbe || nsf > 6144 || nsg > 6144) return LH_EINVAL;
  if (c->ph.source)
    return set_error(c, LH_EUNSUPPORTED, "the hyper-reduced step has no energy source term");
  const Geom& g = c->g;
  if (nsf > g.nv || nsg > g.ne) return LH_EINVAL;
  lh_rom* r = new lh_rom();
  r->ctx = c;
  r->nbv = nbv; r->nbe = nbe; r->nbx = nbx; r->nsf = nsf; r->nsg = nsg;
  auto fail = [&](lh_status st, const char* m) {
    set_error(c, st, r->err.empty() ? m : r->err);
    rom_free(r);
    delete r;
    return st;
  };
  const int64_t NV = g.nv, NE = g.ne, nn = g.nnodes;
  cudaStream_t s = c->stream;
  cudaError_t e = cudaStreamSynchronize(s);
  // host copies of the bases and offsets
  std::vector<double> hv((size_t)NV * nbv), he((size_t)NE * nbe), hx((size_t)NV * nbx);
  std::vector<double> hvos(NV), heos(NE), hxos(NV), rho0K(g.nelem);
  if (e == cudaSuccess) e = cudaMemcpy(hv.data(), Phi_v, hv.size() * 8, cudaMemcpyDefault);
  if (e == cudaSuccess) e = cudaMemcpy(he.data(), Phi_e, he.size() * 8, cudaMemcpyDefault);
  if (e == cudaSuccess) e = cudaMemcpy(hx.data(), Phi_x, hx.size() * 8, cudaMemcpyDefault);
  if (e == cudaSuccess) e = cudaMemcpy(hvos.data(), v_os, NV * 8, cudaMemcpyDefault);
  if (e == cudaSuccess) e = cudaMemcpy(heos.data(), e_os, NE * 8, cudaMemcpyDefault);
  if (e == cudaSuccess) e = cudaMemcpy(hxos.data(), x_os, NV * 8, cudaMemcpyDefault);
  if (e == cudaSuccess) e = cudaMemcpy(rho0K.data(), c->a.rho0K, g.nelem * 8, cudaMemcpyDeviceToHost);
  if (rom_cuda(r, e, "basis copy") != LH_OK) return fail(LH_ECUDA, "basis copy");
  // SNS basis Phi_F = M_V Phi_v on the device (partially assembled operator),
  // essential rows set to zero
  std::vector<double> hF((size_t)NV * nbv);
  {
    double *din = nullptr, *dout = nullptr;
    e = cudaMalloc((void**)&din, NV * 8);
    if (e == cudaSuccess) e = cudaMalloc((void**)&dout, NV * 8);
    for (int j = 0; j < nbv && e == cudaSuccess; ++j) {
      e = cudaMemcpyAsync(din, hv.data() + (size_t)j * NV, NV * 8, cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess) e = launch_mass_apply(c, din, dout, s);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(hF.data() + (size_t)j * NV, dout, NV * 8, cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    if (din) cudaFree(din);
    if (dout) cudaFree(dout);
    if (rom_cuda(r, e, "SNS basis") != LH_OK) return fail(LH_ECUDA, "SNS basis");
    for (int64_t node = 0; node < nn; ++node) {
      int I[3] = {(int)(node % g.nn[0]), (int)((node / g.nn[0]) % g.nn[1]),
                  (int)(node / ((int64_t)g.nn[0] * g.nn[1]))};
      for (int cc = 0; cc < g.dim; ++cc)
        if (I[cc] == 0 || I[cc] == g.nn[cc] - 1)
          for (int j = 0; j < nbv; ++j) hF[(size_t)j * NV + cc * nn + node] = 0.0;
    }
  }
  // SNS basis Phi_G = M_E Phi_e: per element rho0|J0| times the reference L2
  // mass matrix (tensor product of the 1D Gauss-Legendre mass matrices)
  std::vector<double> hG((size_t)NE * nbe);
  {
    const int k = g.k, d = g.dim, nq = g.nq;
    double m1[kMaxOrder][kMaxOrder];
    for (int a = 0; a < k; ++a)
      for (int b = 0; b < k; ++b) {
        double acc = 0.0;
        for (int q = 0; q < nq; ++q) acc += c->basis.W[q] * c->basis.L[q][a] * c->basis.L[q][b];
        m1[a][b] = acc;
      }
    int nd2 = 1;
    for (int i = 0; i < d; ++i) nd2 *= k;
    for (int64_t el = 0; el < g.nelem; ++el)
      for (int i = 0; i < nd2; ++i)
        for (int jb = 0; jb < nbe; ++jb) {
          double acc = 0.0;
          for (int j = 0; j < nd2; ++j) {
            double mij = 1.0;
            int ii = i, jj = j;
            for (int dd = 0; dd < d; ++dd) {
              mij *= m1[ii % k][jj % k];
              ii /= k;
              jj /= k;
            }
            acc += mij * he[(size_t)jb * NE + el * nd2 + j];
          }
          hG[(size_t)jb * NE + el * nd2 + i] = rho0K[el] * acc;
        }
  }
  // sample rows
  if (samples_f) r->hsf.assign(samples_f, samples_f + nsf);
  else if (!deim_select(NV, nbv, nsf, hF, r->hsf)) return fail(LH_EINVAL, "DEIM: rank-deficient F.1 basis");
  if (samples_g) r->hsg.assign(samples_g, samples_g + nsg);
  else if (!deim_select(NE, nbe, nsg, hG, r->hsg)) return fail(LH_EINVAL, "DEIM: rank-deficient F^T v basis");
  {
    std::set<int64_t> uf(r->hsf.begin(), r->hsf.end()), ug(r->hsg.begin(), r->hsg.end());
    if ((int)uf.size() != nsf || (int)ug.size() != nsg || *uf.begin() < 0 || *uf.rbegin() >= NV ||
        *ug.begin() < 0 || *ug.rbegin() >= NE)
      return fail(LH_EINVAL, "sample rows must be distinct and in range");
  }
  // least-squares matrices (Z^T Phi)^+
  std::vector<double> B, AF, AG;
  B.assign((size_t)nsf * nbv, 0.0);
  for (int a = 0; a < nsf; ++a)
    for (int j = 0; j < nbv; ++j) B[(size_t)a * nbv + j] = hF[(size_t)j * NV + r->hsf[a]];
  if (!pinv_qr(nsf, nbv, B, AF)) return fail(LH_EINVAL, "Z_F^T Phi_F is rank-deficient");
  B.assign((size_t)nsg * nbe, 0.0);
  for (int a = 0; a < nsg; ++a)
    for (int j = 0; j < nbe; ++j) B[(size_t)a * nbe + j] = hG[(size_t)j * NE + r->hsg[a]];
  if (!pinv_qr(nsg, nbe, B, AG)) return fail(LH_EINVAL, "Z_G^T Phi_G is rank-deficient");
  // sampled elements
  int nd2 = 1;
  for (int i = 0; i < g.dim; ++i) nd2 *= g.k;
  std::vector<int64_t> enodes;
  {
    std::set<int64_t> snodes;
    for (int64_t row : r->hsf) snodes.insert(row % nn);
    std::set<int32_t> els;
    for (int64_t row : r->hsg) els.insert((int32_t)(row / nd2));
    for (int64_t el = 0; el < g.nelem; ++el) {
      element_nodes(g, el, enodes);
      for (int64_t nd : enodes)
        if (snodes.count(nd)) { els.insert((int32_t)el); break; }
    }
    r->hsel.assign(els.begin(), els.end());
    r->nsel = (int64_t)r->hsel.size();
  }
  // lifted rows: every component of every node of the sampled elements; the
  // energy dofs of the sampled elements
  std::vector<int64_t> rows_v, rows_e;
  {
    std::set<int64_t> nodes;
    for (int32_t el : r->hsel) {
      element_nodes(g, el, enodes);
      nodes.insert(enodes.begin(), enodes.end());
    }
    for (int cc = 0; cc < g.dim; ++cc)
      for (int64_t nd : nodes) rows_v.push_back(cc * nn + nd);
    for (int32_t el : r->hsel)
      for (int j = 0; j < nd2; ++j) rows_e.push_back((int64_t)el * nd2 + j);
  }
  r->nrv = (int64_t)rows_v.size();
  r->nre = (int64_t)rows_e.size();
  std::vector<double> Pv(r->nrv * nbv), Px(r->nrv * nbx), Pe(r->nre * nbe), vos(r->nrv),
      xos(r->nrv), eos(r->nre);
  for (int64_t i = 0; i < r->nrv; ++i) {
    for (int j = 0; j < nbv; ++j) Pv[i * nbv + j] = hv[(size_t)j * NV + rows_v[i]];
    for (int j = 0; j < nbx; ++j) Px[i * nbx + j] = hx[(size_t)j * NV + rows_v[i]];
    vos[i] = hvos[rows_v[i]];
    xos[i] = hxos[rows_v[i]];
  }
  for (int64_t i = 0; i < r->nre; ++i) {
    for (int j = 0; j < nbe; ++j) Pe[i * nbe + j] = he[(size_t)j * NE + rows_e[i]];
    eos[i] = heos[rows_e[i]];
  }
  // gather tables: a sampled F.1 entry (c, node) is the sum of the element
  // rows (slot, c, i) of every sampled element that holds node as local i
  const int nd1 = (int)enodes.size();
  std::vector<int32_t> gf_off(nsf + 1, 0), gf_idx, gg_idx(nsg);
  for (int a = 0; a < nsf; ++a) {
    const int64_t row = r->hsf[a], cc = row / nn, node = row % nn;
    for (int64_t slot = 0; slot < r->nsel; ++slot) {
      element_nodes(g, r->hsel[slot], enodes);
      for (int i = 0; i < nd1; ++i)
        if (enodes[i] == node) gf_idx.push_back((int32_t)(slot * g.dim * nd1 + cc * nd1 + i));
    }
    gf_off[a + 1] = (int32_t)gf_idx.size();
  }
  for (int a = 0; a < nsg; ++a) {
    const int64_t el = r->hsg[a] / nd2, j = r->hsg[a] % nd2;
    const int64_t slot = std::lower_bound(r->hsel.begin(), r->hsel.end(), (int32_t)el) - r->hsel.begin();
    gg_idx[a] = (int32_t)(slot * nd2 + j);
  }
  // position equation: C = Phi_x^T Phi_v, b = Phi_x^T v_os
  std::vector<double> C((size_t)nbx * nbv, 0.0), bx(nbx, 0.0);
  for (int jx = 0; jx < nbx; ++jx) {
    const double* px = hx.data() + (size_t)jx * NV;
    double sb = 0.0;
    for (int64_t i = 0; i < NV; ++i) sb += px[i] * hvos[i];
    bx[jx] = sb;
    for (int jv = 0; jv < nbv; ++jv) {
      const double* pv = hv.data() + (size_t)jv * NV;
      double sc = 0.0;
      for (int64_t i = 0; i < NV; ++i) sc += px[i] * pv[i];
      C[(size_t)jx * nbv + jv] = sc;
    }
  }
  // device arrays
  e = up(&r->sel, r->hsel);
  if (e == cudaSuccess) e = up(&r->rows_v, rows_v);
  if (e == cudaSuccess) e = up(&r->rows_e, rows_e);
  if (e == cudaSuccess) e = up(&r->Pv, Pv);
  if (e == cudaSuccess) e = up(&r->Px, Px);
  if (e == cudaSuccess) e = up(&r->Pe, Pe);
  if (e == cudaSuccess) e = up(&r->vos, vos);
  if (e == cudaSuccess) e = up(&r->xos, xos);
  if (e == cudaSuccess) e = up(&r->eos, eos);
  if (e == cudaSuccess) e = up(&r->AF, AF);
  if (e == cudaSuccess) e = up(&r->AG, AG);
  if (e == cudaSuccess) e = up(&r->gf_off, gf_off);
  if (e == cudaSuccess) e = up(&r->gf_idx, gf_idx);
  if (e == cudaSuccess) e = up(&r->gg_idx, gg_idx);
  if (e == cudaSuccess) e = up(&r->C, C);
  if (e == cudaSuccess) e = up(&r->bx, bx);
  if (e == cudaSuccess) e = up(&r->Phv, hv);
  if (e == cudaSuccess) e = up(&r->Phe, he);
  if (e == cudaSuccess) e = up(&r->Phx, hx);
  if (e == cudaSuccess) e = up(&r->fvos, hvos);
  if (e == cudaSuccess) e = up(&r->feos, heos);
  if (e == cudaSuccess) e = up(&r->fxos, hxos);
  const int64_t nred = 3 * (int64_t)(nbv + nbe + nbx) + 2 * nbv + nbe;
  if (e == cudaSuccess) e = cudaMalloc((void**)&r->red, nred * 8);
  if (e == cudaSuccess) e = cudaMemset(r->red, 0, nred * 8);
  if (e == cudaSuccess) e = cudaMalloc((void**)&r->vF, NV * 8);
  if (e == cudaSuccess) e = cudaMalloc((void**)&r->xF, NV * 8);
  if (e == cudaSuccess) e = cudaMalloc((void**)&r->wF, NV * 8);
  if (e == cudaSuccess) e = cudaMalloc((void**)&r->eF, NE * 8);
  if (e == cudaSuccess) e = cudaMemset(r->vF, 0, NV * 8);
  if (e == cudaSuccess) e = cudaMemset(r->xF, 0, NV * 8);
  if (e == cudaSuccess) e = cudaMemset(r->wF, 0, NV * 8);
  if (e == cudaSuccess) e = cudaMemset(r->eF, 0, NE * 8);
  if (e == cudaSuccess) e = cudaMalloc((void**)&r->F1E, std::max<int64_t>(1, r->nsel * g.dim * nd1) * 8);
  if (e == cudaSuccess) e = cudaMalloc((void**)&r->FTvE, std::max<int64_t>(1, r->nsel * nd2) * 8);
  if (e == cudaSuccess) e = cudaMalloc((void**)&r->ctl, sizeof(Ctl));
  if (e == cudaSuccess) e = cudaMemset(r->ctl, 0, sizeof(Ctl));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&r->ctl_host, sizeof(Ctl));
  if (e == cudaSuccess) e = cudaEventCreate(&r->ev0);
  if (e == cudaSuccess) e = cudaEventCreate(&r->ev1);
  if (rom_cuda(r, e, "allocation") != LH_OK) return fail(LH_ENOMEM, "allocation");
  // reduced coordinates: [vh eh xh][vhn ehn xhn][vh2 eh2 xh2] vbar fh gh
  const int nb = nbv + nbe + nbx;
  r->vh = r->red; r->eh = r->vh + nbv; r->xh = r->eh + nbe;
  r->vhn = r->red + nb; r->ehn = r->vhn + nbv; r->xhn = r->ehn + nbe;
  r->vh2 = r->red + 2 * nb; r->eh2 = r->vh2 + nbv; r->xh2 = r->eh2 + nbe;
  r->vbar = r->red + 3 * nb; r->fh = r->vbar + nbv; r->gh = r->fh + nbv;
  *out = r;
  return LH_OK;
}

extern "C" lh_status lh_rom_destroy(lh_rom* r) {
  if (!r) return LH_OK;
  if (r->ctx && r->ctx->stream) cudaStreamSynchronize(r->ctx->stream);
  rom_free(r);
  delete r;
  return LH_OK;
}

extern "C" const char* lh_rom_last_error(const lh_rom* r) { return r ? r->err.c_str() : "null rom"; }

extern "C" lh_status lh_rom_info(const lh_rom* r, lh_rom_info_t* info, int64_t* samples_f,
                                 int64_t* samples_g, int32_t* elems) {
  if (!r) return LH_EINVAL;
  if (info) {
    info->nb_v = r->nbv;
    info->nb_e = r->nbe;
    info->nb_x = r->nbx;
    info->ns_f = r->nsf;
    info->ns_g = r->nsg;
    info->n_elems = r->nsel;
    info->n_rows_v = r->nrv;
    info->n_rows_e = r->nre;
  }
  if (samples_f) std::copy(r->hsf.begin(), r->hsf.end(), samples_f);
  if (samples_g) std::copy(r->hsg.begin(), r->hsg.end(), samples_g);
  if (elems) std::copy(r->hsel.begin(), r->hsel.end(), elems);
  return LH_OK;
}

extern "C" lh_status lh_rom_set_state(lh_rom* r, const double* vh, const double* eh,
                                      const double* xh, double t, double dt) {
  if (!r || !vh || !eh || !xh) return LH_EINVAL;
  cudaStream_t s = r->ctx->stream;
  cudaError_t e = cudaMemcpyAsync(r->vh, vh, r->nbv * 8, cudaMemcpyDefault, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(r->eh, eh, r->nbe * 8, cudaMemcpyDefault, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(r->xh, xh, r->nbx * 8, cudaMemcpyDefault, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  lh_status st = rom_cuda(r, e, "set_state");
  if (st != LH_OK) return st;
  memset(r->ctl_host, 0, sizeof(Ctl));
  r->ctl_host->t = t;
  r->ctl_host->dt = dt;
  e = cudaMemcpyAsync(r->ctl, r->ctl_host, sizeof(Ctl), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return rom_cuda(r, e, "set_state ctl");
}

extern "C" lh_status lh_rom_get_state(lh_rom* r, double* vh, double* eh, double* xh, double* t,
                                      double* dt) {
  if (!r) return LH_EINVAL;
  cudaStream_t s = r->ctx->stream;
  cudaError_t e = cudaSuccess;
  if (vh) e = cudaMemcpyAsync(vh, r->vh, r->nbv * 8, cudaMemcpyDefault, s);
  if (e == cudaSuccess && eh) e = cudaMemcpyAsync(eh, r->eh, r->nbe * 8, cudaMemcpyDefault, s);
  if (e == cudaSuccess && xh) e = cudaMemcpyAsync(xh, r->xh, r->nbx * 8, cudaMemcpyDefault, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(r->ctl_host, r->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  lh_status st = rom_cuda(r, e, "get_state");
  if (st != LH_OK) return st;
  if (t) *t = r->ctl_host->t;
  if (dt) *dt = r->ctl_host->dt;
  return LH_OK;
}

extern "C" lh_status lh_rom_lift(lh_rom* r, double* v, double* e, double* x) {
  if (!r) return LH_EINVAL;
  const Geom& g = r->ctx->g;
  cudaStream_t s = r->ctx->stream;
  auto blocks = [](int64_t n) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 4096)); };
  if (v) rom_lift_full_kernel<<<blocks(g.nv), 256, 0, s>>>(g.nv, r->nbv, r->Phv, r->fvos, r->vh, v);
  if (e) rom_lift_full_kernel<<<blocks(g.ne), 256, 0, s>>>(g.ne, r->nbe, r->Phe, r->feos, r->eh, e);
  if (x) rom_lift_full_kernel<<<blocks(g.nv), 256, 0, s>>>(g.nv, r->nbx, r->Phx, r->fxos, r->xh, x);
  cudaError_t err = cudaGetLastError();
  if (err == cudaSuccess) err = cudaStreamSynchronize(s);
  return rom_cuda(r, err, "lift");
}

extern "C" lh_status lh_rom_step_fixed(lh_rom* r, double dt, double* tau) {
  if (!r || !(dt > 0.0)) return LH_EINVAL;
  lh_status st = rom_run(r, INFINITY, INT64_MAX, 1, dt, nullptr);
  if (tau) *tau = r->ctl_host->tau_last;
  return st;
}

extern "C" lh_status lh_rom_run_to(lh_rom* r, double t_final, int64_t max_steps,
                                   lh_run_stats* stats) {
  if (!r || !(t_final >= 0.0) || max_steps < 0) return LH_EINVAL;
  float ms = 0.f;
  lh_status st = rom_run(r, t_final, max_steps, 0, 0.0, &ms);
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    const Ctl& h = *r->ctl_host;
    stats->steps = h.steps;
    stats->rejects = h.rejects;
    stats->t = h.t;
    stats->dt = h.dt;
    stats->wall_ms = ms;
  }
  return st;
}
