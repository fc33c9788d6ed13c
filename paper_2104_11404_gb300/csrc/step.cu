// RK2-average time step (eq:RK2-avg), the RK4 step (eq:RK4) and the automatic
// step control of Section 2.2.3, orchestrated on the device.
//
// One attempt is the fixed kernel sequence
//   force(S^n) -> gather -> CG -> v, x half update -> energy half update
//   force(S^{n+1/2}) -> gather -> CG -> v, vbar, x update -> energy update
//   control (accept / redo / grow, single thread) -> commit (if accepted)
// with every scalar (dt, t, tau, accept flag) in a device control block, so the
// sequence is captured once as a CUDA graph and relaunched without host
// synchronisation; the host only polls the control block between batches.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include "control.cuh"

namespace lagh {

__global__ void stage1_update_kernel(int64_t nv, const double* __restrict__ v,
                                     const double* __restrict__ x, const double* __restrict__ a,
                                     double* __restrict__ vh, double* __restrict__ xh,
                                     const Ctl* ctl) {
  pdl_enter();
  if (ctl->done) return;
  const double hdt = 0.5 * ctl->dt_use;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv;
       i += (int64_t)gridDim.x * blockDim.x) {
    double vhalf = v[i] + hdt * a[i];
    vh[i] = vhalf;
    xh[i] = x[i] + hdt * vhalf;
  }
}

__global__ void stage2_update_kernel(int64_t nv, const double* __restrict__ v,
                                     const double* __restrict__ x, const double* __restrict__ a,
                                     double* __restrict__ vn, double* __restrict__ vbar,
                                     double* __restrict__ xn, const Ctl* ctl) {
  pdl_enter();
  if (ctl->done) return;
  const double dt = ctl->dt_use;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv;
       i += (int64_t)gridDim.x * blockDim.x) {
    double v1 = v[i] + dt * a[i];
    double vb = 0.5 * (v[i] + v1);
    vn[i] = v1;
    vbar[i] = vb;
    xn[i] = x[i] + dt * vb;
  }
}

// RK4 stage combination (eq:RK4, eq:RK4coeff).  Stage s (0..3) has produced
// its rates: dv/dt = a (the CG solution), de/dt = erate and dx/dt = vs (the
// stage velocity).  They are added to the weighted sums K with weights 1, 2,
// 2, 1; stages 0..2 then form the next stage state S^n + c dt k_s (c = 1/2,
// 1/2, 1), stage 3 the candidate S^n + dt/6 K.  The next stage state may be
// the arrays the current stage's velocity was read from (element-wise, each
// entry is read before it is written), so no pointer here is restrict.
__global__ void rk4_combine_kernel(int64_t nv, int64_t ne, int s, const double* v, const double* x,
                                   const double* e, const double* a, const double* vs,
                                   const double* erate, double* Kv, double* Kx, double* Ke,
                                   double* vnext, double* xnext, double* enext, const Ctl* ctl) {
  pdl_enter();
  if (ctl->done) return;
  const double dt = ctl->dt_use;
  const double w = (s == 1 || s == 2) ? 2.0 : 1.0;
  const double cdt = (s == 2) ? dt : 0.5 * dt;  // c_{s+1} dt of the next stage
  const double h6 = dt / 6.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += stride) {
    const double ai = a[i], vi = vs[i];
    const double kv = s == 0 ? ai : Kv[i] + w * ai;
    const double kx = s == 0 ? vi : Kx[i] + w * vi;
    if (s < 3) {
      Kv[i] = kv;
      Kx[i] = kx;
      vnext[i] = v[i] + cdt * ai;
      xnext[i] = x[i] + cdt * vi;
    } else {
      vnext[i] = v[i] + h6 * kv;
      xnext[i] = x[i] + h6 * kx;
    }
  }
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ne; i += stride) {
    const double ri = erate[i];
    const double ke = s == 0 ? ri : Ke[i] + w * ri;
    if (s < 3) {
      Ke[i] = ke;
      enext[i] = e[i] + cdt * ri;
    } else {
      enext[i] = e[i] + h6 * ke;
    }
  }
}

__global__ void control_kernel(Ctl* ctl, CtlConsts k) {
  pdl_enter();
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  control_update(ctl, k);
}

__global__ void commit_kernel(int64_t nv, int64_t ne, double* __restrict__ v, double* __restrict__ x,
                              double* __restrict__ e, const double* __restrict__ vn,
                              const double* __restrict__ xn, const double* __restrict__ en,
                              const Ctl* ctl) {
  pdl_enter();
  if (!ctl->accepted) return;
  int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += stride) {
    v[i] = vn[i];
    x[i] = xn[i];
  }
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ne; i += stride) e[i] = en[i];
}

// Start of a run: control constants, counters, first dt_use.
__global__ void begin_kernel(Ctl* ctl, double t_final, long long max_steps, double dt_min,
                             int fixed, double dt_fixed, double* dt_log, long long dt_log_cap,
                             const unsigned long long* est_bits) {
  pdl_enter();
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  control_begin(ctl, t_final, max_steps, dt_min, fixed, dt_fixed, dt_log, dt_log_cap, est_bits);
}

__global__ void set_bits_kernel(unsigned long long* p, unsigned long long v, int* flag) {
  pdl_enter();
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    *p = v;
    if (flag) *flag = 0;
  }
}

static int node_blocks(const lh_ctx* c, int64_t n) {
  int64_t b = (n + 255) / 256;
  int64_t cap = (int64_t)c->num_sms * 8;
  return (int)(b < cap ? (b > 0 ? b : 1) : cap);
}

// CG of one stage: a WHILE graph node when capturing, else an eager loop.
static cudaError_t stage_cg(lh_ctx* c, cudaStream_t s, bool capturing) {
  if (capturing) return cg_solve_capture(c, c->a.rhs, c->a.acc, c->a.ctl, s, c->side);
  int done = 0;
  return cg_solve_eager(c, c->a.rhs, c->a.acc, s, &done);
}

static cudaError_t enqueue_control_commit(lh_ctx* c, cudaStream_t s) {
  Arrays& A = c->a;
  const Geom& g = c->g;
  const bool pdl = c->use_pdl != 0;
  CtlConsts k;
  k.beta1 = c->phys_desc.beta1;
  k.beta2 = c->phys_desc.beta2;
  k.gamma_dt = c->phys_desc.gamma_dt;
  cudaError_t e = launch_k(pdl, control_kernel, dim3(1), dim3(32), 0, s, A.ctl, k);
  if (e != cudaSuccess) return e;
  return launch_k(pdl, commit_kernel, dim3(node_blocks(c, g.nv)), dim3(256), 0, s, g.nv, g.ne, A.v,
                  A.x, A.e, (const double*)A.vn, (const double*)A.xn, (const double*)A.en,
                  (const Ctl*)A.ctl);
}

// Enqueue one attempt of the RK4 step (eq:RK4) on stream s: four stages of
// force -> gather -> CG -> energy rate -> combination, then control and commit.
static cudaError_t enqueue_attempt_rk4(lh_ctx* c, cudaStream_t s, bool capturing) {
  Arrays& A = c->a;
  const Geom& g = c->g;
  const bool mixed = c->precision == LH_MIXED;
  const bool pdl = c->use_pdl != 0;
  cudaError_t e;
  for (int st = 0; st < 4; ++st) {
    const double* vs = st == 0 ? A.v : A.vh;
    const double* es = st == 0 ? A.e : A.eh;
    const double* xs = st == 0 ? A.x : A.xh;
    ForceArgs f = {};
    f.v = vs; f.e = es; f.x = xs; f.vtest = nullptr;
    f.list = nullptr; f.nslots = g.nelem;
    f.F1E = A.F1E;
    f.D = mixed ? nullptr : A.D;
    f.FK = mixed ? A.FK : nullptr;
    f.FTvE = nullptr;
    f.srcE = c->ph.source ? A.srcE : nullptr;
    f.tau_bits = &A.ctl->tau_bits[st == 0 ? 0 : 1];  // the minimum over all stages
    f.status = &A.ctl->status;
    f.ctl = A.ctl;
    f.p_ref = &A.ctl->p_ref;
    f.mode = kForceFull;
    if ((e = launch_force(c, f, s)) != cudaSuccess) return e;
    if ((e = launch_gather(c, A.F1E, A.rhs, -1.0, 1, A.ctl, s)) != cudaSuccess) return e;
    if ((e = stage_cg(c, s, capturing)) != cudaSuccess) return e;
    EnergyArgs ea = {};
    ea.w = vs; ea.D = A.D; ea.FK = A.FK;
    ea.srcE = c->ph.source ? A.srcE : nullptr;
    ea.x = mixed ? xs : nullptr;
    ea.p_ref = mixed ? &A.ctl->p_ref : nullptr;
    ea.e_base = nullptr; ea.e_out = A.erate; ea.frac = 1.0; ea.dt = 0.0; ea.rate = 1;
    ea.ctl = A.ctl;
    ea.rho0Kinv = A.rho0Kinv;
    if ((e = launch_energy_update(c, ea, s)) != cudaSuccess) return e;
    double* vnext = st < 3 ? A.vh : A.vn;
    double* xnext = st < 3 ? A.xh : A.xn;
    double* enext = st < 3 ? A.eh : A.en;
    e = launch_k(pdl, rk4_combine_kernel, dim3(node_blocks(c, g.nv)), dim3(256), 0, s, g.nv, g.ne,
                 st, (const double*)A.v, (const double*)A.x, (const double*)A.e,
                 (const double*)A.acc, vs, (const double*)A.erate, A.Kv, A.Kx, A.Ke, vnext, xnext,
                 enext, (const Ctl*)A.ctl);
    if (e != cudaSuccess) return e;
  }
  return enqueue_control_commit(c, s);
}

// Enqueue one attempt of the RK2-average step on stream s.
static cudaError_t enqueue_attempt(lh_ctx* c, cudaStream_t s, bool capturing) {
  if (c->phys_desc.integrator == LH_RK4) return enqueue_attempt_rk4(c, s, capturing);
  Arrays& A = c->a;
  const Geom& g = c->g;
  const bool mixed = c->precision == LH_MIXED;
  cudaError_t e;
  // stage 1: forces of S^n
  ForceArgs f1 = {};
  f1.v = A.v; f1.e = A.e; f1.x = A.x; f1.vtest = nullptr;
  f1.list = nullptr; f1.nslots = g.nelem;
  f1.F1E = A.F1E;
  f1.D = mixed ? nullptr : A.D;
  f1.FK = mixed ? A.FK : nullptr;
  f1.FTvE = nullptr;
  f1.srcE = c->ph.source ? A.srcE : nullptr;
  f1.tau_bits = &A.ctl->tau_bits[0];
  f1.status = &A.ctl->status;
  f1.ctl = A.ctl;
  f1.p_ref = &A.ctl->p_ref;
  f1.mode = kForceFull;
  if ((e = launch_force(c, f1, s)) != cudaSuccess) return e;
  if ((e = launch_gather(c, A.F1E, A.rhs, -1.0, 1, A.ctl, s)) != cudaSuccess) return e;
  if ((e = stage_cg(c, s, capturing)) != cudaSuccess) return e;
  const bool pdl = c->use_pdl != 0;
  e = launch_k(pdl, stage1_update_kernel, dim3(node_blocks(c, g.nv)), dim3(256), 0, s, g.nv, A.v,
               A.x, A.acc, A.vh, A.xh, A.ctl);
  if (e != cudaSuccess) return e;
  EnergyArgs e1 = {};
  e1.w = A.vh; e1.D = A.D; e1.FK = A.FK;
  e1.srcE = c->ph.source ? A.srcE : nullptr;
  e1.x = mixed ? A.x : nullptr;  // the reference-pressure term uses the force's state
  e1.p_ref = mixed ? &A.ctl->p_ref : nullptr;
  e1.e_base = A.e; e1.e_out = A.eh; e1.frac = 0.5; e1.dt = 0.0; e1.ctl = A.ctl;
  e1.rho0Kinv = A.rho0Kinv;
  if ((e = launch_energy_update(c, e1, s)) != cudaSuccess) return e;
  // stage 2: forces of S^{n+1/2}
  ForceArgs f2 = f1;
  f2.v = A.vh; f2.e = A.eh; f2.x = A.xh;
  f2.tau_bits = &A.ctl->tau_bits[1];
  if ((e = launch_force(c, f2, s)) != cudaSuccess) return e;
  if ((e = launch_gather(c, A.F1E, A.rhs, -1.0, 1, A.ctl, s)) != cudaSuccess) return e;
  if ((e = stage_cg(c, s, capturing)) != cudaSuccess) return e;
  e = launch_k(pdl, stage2_update_kernel, dim3(node_blocks(c, g.nv)), dim3(256), 0, s, g.nv, A.v,
               A.x, A.acc, A.vn, A.vbar, A.xn, A.ctl);
  if (e != cudaSuccess) return e;
  EnergyArgs e2 = e1;
  e2.w = A.vbar; e2.e_out = A.en; e2.frac = 1.0;
  e2.x = mixed ? A.xh : nullptr;
  if ((e = launch_energy_update(c, e2, s)) != cudaSuccess) return e;
  return enqueue_control_commit(c, s);
}

static cudaError_t capture_attempt(lh_ctx* c, const char** where) {
  cudaGraph_t graph = nullptr;
  *where = "begin capture";
  cudaError_t e = cudaStreamBeginCapture(c->work, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaError_t e2 = enqueue_attempt(c, c->work, true);
    *where = "enqueue";
    e = cudaStreamEndCapture(c->work, &graph);
    if (e2 != cudaSuccess) e = e2;
    else *where = "end capture";
  }
  if (e == cudaSuccess) {
    *where = "instantiate";
    e = cudaGraphInstantiate(&c->step_graph, graph, 0);
  }
  if (graph) cudaGraphDestroy(graph);
  if (e != cudaSuccess) cudaGetLastError();
  return e;
}

static lh_status build_graph(lh_ctx* c) {
  if (c->graph_ready != 0) return LH_OK;
  if (c->phys_desc.direct_launch) {
    c->graph_ready = -1;
    return LH_OK;
  }
  const char* where = "";
  cudaError_t e = capture_attempt(c, &where);
  if (e != cudaSuccess && c->use_pdl) {  // retry without programmatic dependent launch
    c->use_pdl = 0;
    e = capture_attempt(c, &where);
  }
  if (e != cudaSuccess && c->cg_cluster > 0) {  // and with the CG as a kernel chain
    c->cg_cluster = 0;
    e = capture_attempt(c, &where);
  }
  if (e == cudaSuccess) {
    c->graph_ready = 1;
  } else {
    c->graph_ready = -1;  // capture not available: launch the sequence eagerly
    fprintf(stderr, "lagh: step graph not built at %s (%s); launching kernels directly\n",
            where, cudaGetErrorString(e));
  }
  return LH_OK;
}

static cudaError_t launch_attempt(lh_ctx* c) {
  if (c->graph_ready == 1) return cudaGraphLaunch(c->step_graph, c->work);
  return enqueue_attempt(c, c->work, false);
}

// Orders the work stream after the user stream (and back at the end).
static cudaError_t join_work(lh_ctx* c, bool to_work) {
  if (c->work == c->stream) return cudaSuccess;
  cudaEvent_t ev = c->ev1;
  if (to_work) {
    cudaError_t e = cudaEventRecord(ev, c->stream);
    return e == cudaSuccess ? cudaStreamWaitEvent(c->work, ev, 0) : e;
  }
  cudaError_t e = cudaEventRecord(ev, c->work);
  return e == cudaSuccess ? cudaStreamWaitEvent(c->stream, ev, 0) : e;
}

static lh_status read_ctl(lh_ctx* c, cudaStream_t s) {
  cudaError_t e = cudaMemcpyAsync(c->ctl_host, c->a.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return cuda_check(c, e, "read control block");
}

// Estimate of the current state into aux[0] (ordered bits).
static cudaError_t estimate_into_aux(lh_ctx* c, cudaStream_t s) {
  unsigned long long* bits = reinterpret_cast<unsigned long long*>(c->a.aux);
  int* flag = reinterpret_cast<int*>(c->a.aux + 1);
  set_bits_kernel<<<1, 32, 0, s>>>(bits, kInfBits, flag);
  ForceArgs f = {};
  f.v = c->a.v; f.e = c->a.e; f.x = c->a.x;
  f.nslots = c->g.nelem;
  f.F1E = c->a.F1E;
  f.tau_bits = bits;
  f.status = flag;
  f.p_ref = &c->a.ctl->p_ref;
  return launch_force(c, f, s);
}

static lh_status status_from(lh_ctx* c, int s) {
  if (s & kDevNonFinite) return set_error(c, LH_ENONFINITE, "non-finite value in the state");
  if (s & kDevCG) return set_error(c, LH_ECG, "CG did not converge within cg_maxit");
  if (s & kDevDtMin) return set_error(c, LH_EDTMIN, "time step collapsed below dt_min");
  return LH_OK;
}

// Common driver of lh_run_to / lh_step / lh_step_fixed.
static lh_status run_attempts(lh_ctx* c, double t_final, int64_t max_steps, int fixed,
                              double dt_fixed, int64_t max_attempts, double* dt_log,
                              int64_t dt_log_cap, float* wall_ms) {
  lh_status st = build_graph(c);
  if (st != LH_OK) return st;
  cudaError_t e = join_work(c, true);
  if ((st = cuda_check(c, e, "stream join")) != LH_OK) return st;
  if ((st = read_ctl(c, c->work)) != LH_OK) return st;
  if (!fixed && !(c->ctl_host->dt > 0.0)) {
    if ((st = cuda_check(c, estimate_into_aux(c, c->work), "initial estimate")) != LH_OK) return st;
  }
  begin_kernel<<<1, 32, 0, c->work>>>(c->a.ctl, t_final, (long long)max_steps,
                                      c->phys_desc.dt_min_frac * t_final, fixed, dt_fixed, dt_log,
                                      (long long)dt_log_cap,
                                      reinterpret_cast<const unsigned long long*>(c->a.aux));
  if ((st = cuda_check(c, cudaGetLastError(), "begin")) != LH_OK) return st;
  if ((st = read_ctl(c, c->work)) != LH_OK) return st;
  cudaEventRecord(c->ev0, c->work);
  int64_t attempts = 0;
  while (!c->ctl_host->done && attempts < max_attempts) {
    // launch a batch sized by the remaining time, then poll the control block
    const Ctl& h = *c->ctl_host;
    int64_t batch = 1;
    if (!fixed && h.dt > 0.0) {
      double rem = (h.t_final - h.t) / h.dt;
      batch = rem > 64.0 ? 64 : (int64_t)rem + 1;
      // a few attempts beyond the remaining step budget absorb redone steps
      int64_t left = h.max_steps - h.steps + 2;
      if (left < batch) batch = left > 1 ? left : 1;
    }
    if (batch > max_attempts - attempts) batch = max_attempts - attempts;
    for (int64_t i = 0; i < batch; ++i) {
      e = launch_attempt(c);
      if ((st = cuda_check(c, e, "step launch")) != LH_OK) return st;
    }
    attempts += batch;
    if ((st = read_ctl(c, c->work)) != LH_OK) return st;
  }
  cudaEventRecord(c->ev1, c->work);
  e = cudaEventSynchronize(c->ev1);
  if ((st = cuda_check(c, e, "run sync")) != LH_OK) return st;
  if (wall_ms) cudaEventElapsedTime(wall_ms, c->ev0, c->ev1);
  if ((st = read_ctl(c, c->work)) != LH_OK) return st;
  if ((st = cuda_check(c, join_work(c, false), "stream join")) != LH_OK) return st;
  return status_from(c, c->ctl_host->status);
}

}  // namespace lagh

using namespace lagh;

extern "C" lh_status lh_run_to(lh_ctx* c, double t_final, int64_t max_steps, lh_run_stats* stats,
                               double* dt_log, int64_t dt_log_cap) {
  if (!c || !(t_final >= 0.0) || max_steps < 0) return LH_EINVAL;
  lh_status st;
  double E0 = 0.0;
  if (stats && (st = lh_total_energy(c, &E0)) != LH_OK) return st;
  float ms = 0.f;
  st = run_attempts(c, t_final, max_steps, 0, 0.0, INT64_MAX, dt_log, dt_log ? dt_log_cap : 0, &ms);
  if (stats) {
    const Ctl& h = *c->ctl_host;
    stats->steps = h.steps;
    stats->rejects = h.rejects;
    stats->cg_iters = h.cg_iters;
    stats->t = h.t;
    stats->dt = h.dt;
    stats->energy0 = E0;
    stats->wall_ms = ms;
    double E1 = 0.0;
    if (st == LH_OK) {
      lh_status s2 = lh_total_energy(c, &E1);
      if (s2 != LH_OK) return s2;
    }
    stats->energy = E1;
  }
  return st;
}

extern "C" lh_status lh_step(lh_ctx* c, double t_final, int32_t* accepted, double* t, double* dt) {
  if (!c) return LH_EINVAL;
  lh_status st = run_attempts(c, t_final, INT64_MAX, 0, 0.0, 1, nullptr, 0, nullptr);
  const Ctl& h = *c->ctl_host;
  if (accepted) *accepted = h.accepted;
  if (t) *t = h.t;
  if (dt) *dt = h.dt;
  return st;
}

extern "C" lh_status lh_step_fixed(lh_ctx* c, double dt, double* tau) {
  if (!c || !(dt > 0.0)) return LH_EINVAL;
  lh_status st = run_attempts(c, INFINITY, INT64_MAX, 1, dt, 1, nullptr, 0, nullptr);
  if (tau) *tau = c->ctl_host->tau_last;
  // the replay mode is left for the next call; dt is kept as the proposal
  return st;
}

extern "C" lh_status lh_force(lh_ctx* c, const double* v, const double* e, const double* x,
                              const double* vtest, double* F1, double* FTv, double* dt_est) {
  if (!c || !v || !e || !x || !F1) return LH_EINVAL;
  if (vtest && !FTv) return LH_EINVAL;
  cudaStream_t s = c->stream;
  unsigned long long* bits = reinterpret_cast<unsigned long long*>(c->a.aux);
  int* flag = reinterpret_cast<int*>(c->a.aux + 1);
  set_bits_kernel<<<1, 32, 0, s>>>(bits, kInfBits, flag);
  ForceArgs f = {};
  f.v = v; f.e = e; f.x = x; f.vtest = vtest;
  f.nslots = c->g.nelem;
  f.F1E = c->a.F1E;
  f.FTvE = vtest ? FTv : nullptr;
  f.tau_bits = bits;
  f.status = flag;
  f.p_ref = &c->a.ctl->p_ref;
  lh_status st = cuda_check(c, launch_force(c, f, s), "force");
  if (st != LH_OK) return st;
  if (c->precision == LH_MIXED && vtest) {
    // add F^T vtest of the reference pressure left out of the FP32 stress; its
    // F.1 part vanishes identically after the wall condition on the box
    ForceArgs r = f;
    r.F1E = nullptr;
    r.tau_bits = nullptr;
    r.status = nullptr;
    r.mode = kForceRefPressure;
    r.accumulate = 1;
    if ((st = cuda_check(c, launch_force_fp64(c, r, s), "force ref")) != LH_OK) return st;
  }
  st = cuda_check(c, launch_gather(c, c->a.F1E, F1, 1.0, 1, nullptr, s), "gather");
  if (st != LH_OK) return st;
  if (dt_est) {
    double hb[2];
    cudaError_t err = cudaMemcpyAsync(hb, c->a.aux, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (err == cudaSuccess) err = cudaStreamSynchronize(s);
    if ((st = cuda_check(c, err, "force estimate")) != LH_OK) return st;
    unsigned long long b;
    memcpy(&b, &hb[0], 8);
    double tau;
    memcpy(&tau, &b, 8);
    *dt_est = tau;
    int fl;
    memcpy(&fl, &hb[1], sizeof(int));
    if (fl & kDevNonFinite) return set_error(c, LH_ENONFINITE, "non-finite value in the state");
    if (fl & kDevTangled) return set_error(c, LH_ETANGLED, "inverted element (|J| <= 0)");
  }
  return LH_OK;
}

extern "C" lh_status lh_force_sampled(lh_ctx* c, const int32_t* elem_ids, int64_t n,
                                      const double* v, const double* e, const double* x,
                                      const double* vtest, double* F1_local, double* FTv_local,
                                      double* dt_est) {
  if (!c || n < 0 || !v || !e || !x || (n > 0 && (!elem_ids || !F1_local))) return LH_EINVAL;
  if (vtest && !FTv_local) return LH_EINVAL;
  cudaStream_t s = c->stream;
  unsigned long long* bits = reinterpret_cast<unsigned long long*>(c->a.aux);
  int* flag = reinterpret_cast<int*>(c->a.aux + 1);
  set_bits_kernel<<<1, 32, 0, s>>>(bits, kInfBits, flag);
  ForceArgs f = {};
  f.v = v; f.e = e; f.x = x; f.vtest = vtest;
  f.list = elem_ids;
  f.nslots = n;
  f.F1E = F1_local;
  f.FTvE = vtest ? FTv_local : nullptr;
  f.tau_bits = bits;
  f.status = flag;
  f.p_ref = &c->a.ctl->p_ref;
  lh_status st = cuda_check(c, launch_force(c, f, s), "force_sampled");
  if (st != LH_OK) return st;
  if (c->precision == LH_MIXED && n > 0) {
    // element rows carry no wall condition: add the reference-pressure part
    ForceArgs r = f;
    r.tau_bits = nullptr;
    r.status = nullptr;
    r.mode = kForceRefPressure;
    r.accumulate = 1;
    if ((st = cuda_check(c, launch_force_fp64(c, r, s), "force_sampled ref")) != LH_OK) return st;
  }
  if (dt_est) {
    double hb[2];
    cudaError_t err = cudaMemcpyAsync(hb, c->a.aux, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (err == cudaSuccess) err = cudaStreamSynchronize(s);
    if ((st = cuda_check(c, err, "sampled estimate")) != LH_OK) return st;
    double tau;
    memcpy(&tau, &hb[0], 8);
    *dt_est = tau;
    int fl;
    memcpy(&fl, &hb[1], sizeof(int));
    if (fl & kDevNonFinite) return set_error(c, LH_ENONFINITE, "non-finite value in the state");
    if (fl & kDevTangled) return set_error(c, LH_ETANGLED, "inverted element (|J| <= 0)");
  }
  return LH_OK;
}

extern "C" lh_status lh_mass_apply_v(lh_ctx* c, const double* in, double* out) {
  if (!c || !in || !out) return LH_EINVAL;
  return cuda_check(c, launch_mass_apply(c, in, out, c->stream), "mass apply");
}

extern "C" lh_status lh_mass_solve_v(lh_ctx* c, const double* rhs, double* out, int32_t* iters,
                                     double* relres) {
  if (!c || !rhs || !out) return LH_EINVAL;
  int done = 0;
  lh_status st = cuda_check(c, cg_solve_eager(c, rhs, out, c->stream, &done), "cg");
  if (st != LH_OK) return st;
  if (iters || relres) {
    if ((st = read_ctl(c, c->stream)) != LH_OK) return st;
    if (iters) *iters = c->ctl_host->cg_last_iters;
    if (relres) *relres = c->ctl_host->cg_last_relres;
    int s = c->ctl_host->status;
    if (s & (kDevCG | kDevTimeout)) {
      // report once and clear, the solve does not poison the time loop state
      int clear = 0;
      cudaMemcpyAsync(&c->a.ctl->status, &clear, sizeof(int), cudaMemcpyHostToDevice, c->stream);
      cudaStreamSynchronize(c->stream);
      return status_from(c, s & (kDevCG | kDevTimeout));
    }
  }
  return LH_OK;
}

extern "C" lh_status lh_precond_apply(lh_ctx* c, const double* in, double* out) {
  if (!c || !in || !out) return LH_EINVAL;
  if (!c->tpc.enabled) return set_error(c, LH_EUNSUPPORTED, "context uses the Jacobi preconditioner");
  return cuda_check(c, precond_apply(c, in, out, c->stream), "precond apply");
}

extern "C" lh_status lh_mass_solve_e(lh_ctx* c, const double* rhs, double* out) {
  if (!c || !rhs || !out) return LH_EINVAL;
  return cuda_check(c, launch_mass_solve_e(c, rhs, out, c->stream), "mass solve e");
}

extern "C" lh_status lh_total_energy(lh_ctx* c, double* energy) {
  if (!c || !energy) return LH_EINVAL;
  cudaStream_t s = c->stream;
  lh_status st = cuda_check(c, launch_total_energy(c, c->a.v, c->a.e, c->a.aux + 2, s), "energy");
  if (st != LH_OK) return st;
  cudaError_t err = cudaMemcpyAsync(energy, c->a.aux + 2, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (err == cudaSuccess) err = cudaStreamSynchronize(s);
  return cuda_check(c, err, "energy");
}
