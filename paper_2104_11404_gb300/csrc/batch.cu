// Host side of the batched form (see batch_kernels.cuh for the device side):
// instance descriptors and packed arrays, the attempt graph (stage 0 kernel,
// stage 1 kernel), the run loop, the autotuner of the launch shape and the
// batched restricted force.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <vector>

#include "batch_kernels.cuh"

namespace lagh {

// Launch shapes built per (dim, order, precision): threads per CTA.
static const int kThreadChoices[3] = {256, 512, 1024};

static bool get_ops(int dim, int k, bool mixed, int ntt, int qpt, BOps* out) {
  if (dim == 3) return get_batch_ops_3d(k, mixed, ntt, qpt, out);
  return qpt == 2 ? get_batch_ops_2d_q2(k, mixed, ntt, qpt, out)
                  : get_batch_ops_2d_q1(k, mixed, ntt, qpt, out);
}

}  // namespace lagh

using namespace lagh;

struct lh_batch {
  int n = 0, dim = 0, k = 0, precision = 0;
  cudaStream_t stream = nullptr;  // user stream
  cudaStream_t work = nullptr;    // capture / launch stream
  int own_work = 0;
  int num_sms = 0;
  size_t smem_optin = 0;
  Basis1D basis;
  std::vector<BInst> inst;
  std::vector<lh_phys_desc> phys;
  std::vector<int64_t> off_v, off_e, off_el;
  int64_t tot_v = 0, tot_e = 0, tot_el = 0;
  int64_t max_nelem = 0, max_nv = 0, max_ne = 0, max_nnodes = 0;
  int has_source = 0;
  double rtol = 1e-14;
  int maxit = 100;
  // device memory
  BInst* d_inst = nullptr;
  int32_t* d_order = nullptr;
  Ctl* d_ctl = nullptr;
  double *v = nullptr, *e = nullptr, *x = nullptr, *vh = nullptr, *eh = nullptr, *xh = nullptr;
  double *vn = nullptr, *en = nullptr, *xn = nullptr, *vbar = nullptr;
  double* rho0K = nullptr;
  double* rho0Kinv = nullptr;
  double* fac = nullptr;
  double* F1E = nullptr;
  float* FK = nullptr;
  double* D = nullptr;
  double* srcE = nullptr;
  double* vec = nullptr;
  double* aux = nullptr;  // n doubles: estimates, energies, fixed step sizes
  unsigned int* qctr = nullptr;
  int* ndone = nullptr;
  // snapshot capture (caller-owned matrices; offsets and counts are ours)
  double *Sv = nullptr, *Se = nullptr, *Sx = nullptr;
  int64_t snap_cap = 0;
  int64_t* d_snap_ov = nullptr;  // n + n offsets (v/x then e) followed by n counts
  int snap_on = 0;
  int64_t s_f1e = 0, s_fkd = 0, s_src = 0, s_vec = 0;
  int slots = 0;
  // host mirrors
  Ctl* ctl_host = nullptr;  // pinned, n entries
  int* ndone_host = nullptr;
  // launch shape
  lh_batch_tuning tune;
  int tuned = 0;       // 1: chosen by the autotuner or fixed by the caller
  BOps ops;
  size_t stage_smem = 0;
  cudaGraphExec_t graph = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  std::string err;
};

namespace lagh {

static lh_status bset_error(lh_batch* b, lh_status s, const std::string& m) {
  b->err = m;
  return s;
}

static lh_status bcheck(lh_batch* b, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return LH_OK;
  return bset_error(b, LH_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

static BatchArgs bargs(const lh_batch* b) {
  BatchArgs a;
  memset(&a, 0, sizeof(a));
  a.inst = b->d_inst;
  a.order = b->d_order;
  a.n = b->n;
  a.ctl = b->d_ctl;
  a.v = b->v; a.e = b->e; a.x = b->x;
  a.vh = b->vh; a.eh = b->eh; a.xh = b->xh;
  a.vn = b->vn; a.en = b->en; a.xn = b->xn;
  a.vbar = b->vbar;
  a.rho0K = b->rho0K;
  a.rho0Kinv = b->rho0Kinv;
  a.fac = b->fac;
  a.F1E = b->F1E;
  a.FK = b->FK;
  a.D = b->D;
  a.srcE = b->srcE;
  a.vec = b->vec;
  a.s_f1e = b->s_f1e;
  a.s_fkd = b->s_fkd;
  a.s_src = b->s_src;
  a.s_vec = b->s_vec;
  a.qctr = b->qctr;
  a.ndone = b->ndone;
  a.rtol = b->rtol;
  a.maxit = b->maxit;
  a.smem_lines = b->tune.smem_lines;
  if (b->snap_on) {
    a.Sv = b->Sv;
    a.Se = b->Se;
    a.Sx = b->Sx;
    a.snap_ov = b->d_snap_ov;
    a.snap_oe = b->d_snap_ov + b->n;
    a.snap_count = b->d_snap_ov + 2 * b->n;
    a.snap_cap = b->snap_cap;
  }
  return a;
}

static int grid_of(const lh_batch* b) {
  int g = b->num_sms * (b->tune.ctas_per_sm > 0 ? b->tune.ctas_per_sm : 1);
  return g < b->slots ? g : b->slots;
}

static int aux_grid(const lh_batch* b) { return b->slots < b->n ? b->slots : b->n; }

static cudaError_t set_smem(const void* fn, size_t bytes) {
  return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Selects a launch shape: ops, shared memory and attributes.  Fails if the
// shape does not fit the device.
static lh_status apply_tuning(lh_batch* b, const lh_batch_tuning& t) {
  BOps o;
  if (!get_ops(b->dim, b->k, b->precision == LH_MIXED, t.threads, t.qpt > 0 ? t.qpt : 1, &o))
    return bset_error(b, LH_EUNSUPPORTED, "launch shape not built for this dimension and order");
  const size_t bytes = o.stage_bytes(b->max_nnodes, t.smem_lines);
  if (bytes > b->smem_optin)
    return bset_error(b, LH_EUNSUPPORTED, "launch shape needs more shared memory than a CTA has");
  cudaError_t e = set_smem(o.stage, bytes);
  if (e == cudaSuccess) e = set_smem(o.estimate, bytes);
  if (e == cudaSuccess) e = set_smem(o.sampled, bytes);
  if (e == cudaSuccess) e = set_smem(o.energy, o.energy_bytes);
  lh_status st = bcheck(b, e, "kernel attributes");
  if (st != LH_OK) return st;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, o.stage, t.threads, bytes);
  if ((st = bcheck(b, e, "occupancy")) != LH_OK) return st;
  if (occ < 1) return bset_error(b, LH_EUNSUPPORTED, "launch shape does not fit an SM");
  lh_batch_tuning tt = t;
  if (tt.ctas_per_sm <= 0 || tt.ctas_per_sm > occ) tt.ctas_per_sm = occ;
  tt.qpt = o.qpt;
  b->ops = o;
  b->stage_smem = bytes;
  b->tune = tt;
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  return LH_OK;
}

static cudaError_t launch_stage(lh_batch* b, int stage, cudaStream_t s) {
  BatchArgs a = bargs(b);
  int st = stage;
  void* args[] = {&a, &b->basis, &st};
  return cudaLaunchKernel(b->ops.stage, dim3(grid_of(b)), dim3(b->tune.threads), args,
                          b->stage_smem, s);
}

// Attempt graph: stage 0 kernel -> stage 1 kernel.
static lh_status build_graph(lh_batch* b) {
  if (b->graph) return LH_OK;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(b->work, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaError_t e1 = launch_stage(b, 0, b->work);
    cudaError_t e2 = e1 == cudaSuccess ? launch_stage(b, 1, b->work) : e1;
    e = cudaStreamEndCapture(b->work, &g);
    if (e2 != cudaSuccess) e = e2;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, g, 0);
  if (g) cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    b->graph = nullptr;
    return bcheck(b, e, "attempt graph");
  }
  return LH_OK;
}

static cudaError_t join(lh_batch* b, bool to_work) {
  if (b->work == b->stream) return cudaSuccess;
  cudaEvent_t ev = b->ev1;
  cudaStream_t from = to_work ? b->stream : b->work, to = to_work ? b->work : b->stream;
  cudaError_t e = cudaEventRecord(ev, from);
  return e == cudaSuccess ? cudaStreamWaitEvent(to, ev, 0) : e;
}

__global__ void batch_begin_kernel(Ctl* ctl, const BInst* inst, int n, double t_final,
                                   long long max_steps, int fixed, const double* aux,
                                   const double* dt_min_frac, int* ndone) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const unsigned long long* est = reinterpret_cast<const unsigned long long*>(aux);
  control_begin(ctl + i, t_final, max_steps, dt_min_frac[i] * t_final, fixed,
                fixed ? aux[i] : 0.0, nullptr, 0, est + i);
  if (ctl[i].done) atomicAdd(ndone, 1);
}

static lh_status read_ctl(lh_batch* b) {
  cudaError_t e = cudaMemcpyAsync(b->ctl_host, b->d_ctl, sizeof(Ctl) * b->n,
                                  cudaMemcpyDeviceToHost, b->work);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->work);
  return bcheck(b, e, "read control blocks");
}

static lh_status instance_status(lh_batch* b) {
  for (int i = 0; i < b->n; ++i) {
    const int s = b->ctl_host[i].status;
    char buf[96];
    if (s & kDevNonFinite) {
      snprintf(buf, sizeof buf, "instance %d: non-finite value in the state", i);
      return bset_error(b, LH_ENONFINITE, buf);
    }
    if (s & kDevCG) {
      snprintf(buf, sizeof buf, "instance %d: CG did not converge within cg_maxit", i);
      return bset_error(b, LH_ECG, buf);
    }
    if (s & kDevDtMin) {
      snprintf(buf, sizeof buf, "instance %d: time step collapsed below dt_min", i);
      return bset_error(b, LH_EDTMIN, buf);
    }
  }
  return LH_OK;
}

static lh_status launch_aux(lh_batch* b, const void* fn, size_t smem, BatchArgs& a,
                            void* extra, cudaStream_t s) {
  cudaError_t e;
  if (extra) {
    void* args[] = {&a, &b->basis, extra};
    e = cudaLaunchKernel(fn, dim3(aux_grid(b)), dim3(b->tune.threads), args, smem, s);
  } else {
    void* args[] = {&a, &b->basis};
    e = cudaLaunchKernel(fn, dim3(aux_grid(b)), dim3(b->tune.threads), args, smem, s);
  }
  return bcheck(b, e, "batched kernel launch");
}

// Estimates of the current states into aux (ordered bits) and run start.
static lh_status begin_run(lh_batch* b, double t_final, int64_t max_steps, int fixed,
                           const double* dt_fixed_host) {
  lh_status st;
  cudaError_t e = cudaMemsetAsync(b->ndone, 0, sizeof(int), b->work);
  if ((st = bcheck(b, e, "reset")) != LH_OK) return st;
  if (fixed) {
    e = cudaMemcpyAsync(b->aux, dt_fixed_host, sizeof(double) * b->n, cudaMemcpyHostToDevice,
                        b->work);
    if ((st = bcheck(b, e, "step sizes")) != LH_OK) return st;
  } else {
    if ((st = read_ctl(b)) != LH_OK) return st;
    bool need = false;
    for (int i = 0; i < b->n && !need; ++i) need = !(b->ctl_host[i].dt > 0.0);
    if (need) {
      BatchArgs a = bargs(b);
      a.out = b->aux;
      if ((st = launch_aux(b, b->ops.estimate, b->stage_smem, a, nullptr, b->work)) != LH_OK)
        return st;
    }
  }
  // per-instance dt_min fractions live after the estimates
  double* frac = b->aux + b->n;
  std::vector<double> fr(b->n);
  for (int i = 0; i < b->n; ++i) fr[i] = b->phys[i].dt_min_frac;
  e = cudaMemcpyAsync(frac, fr.data(), sizeof(double) * b->n, cudaMemcpyHostToDevice, b->work);
  if ((st = bcheck(b, e, "dt_min")) != LH_OK) return st;
  batch_begin_kernel<<<(b->n + 127) / 128, 128, 0, b->work>>>(b->d_ctl, b->d_inst, b->n, t_final,
                                                             (long long)max_steps, fixed, b->aux,
                                                             frac, b->ndone);
  // fr must outlive the copy
  e = cudaStreamSynchronize(b->work);
  return bcheck(b, e == cudaSuccess ? cudaGetLastError() : e, "begin");
}

// Launches attempt graphs until every instance is done: first a batch sized
// by the step budget (a run of a few steps needs no poll in between), then
// growing batches with a poll of the finished count before each.
static lh_status run_loop(lh_batch* b, int64_t max_attempts, int64_t first_batch, float* wall_ms,
                          int64_t* launched) {
  lh_status st;
  if ((st = build_graph(b)) != LH_OK) return st;
  cudaEventRecord(b->ev0, b->work);
  int64_t att = 0;
  int64_t batch = first_batch > 0 ? first_batch : 4;
  cudaError_t e = cudaSuccess;
  while (att < max_attempts) {
    e = cudaMemcpyAsync(b->ndone_host, b->ndone, sizeof(int), cudaMemcpyDeviceToHost, b->work);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->work);
    if ((st = bcheck(b, e, "poll")) != LH_OK) return st;
    if (*b->ndone_host >= b->n) break;
    int64_t nb = batch < max_attempts - att ? batch : max_attempts - att;
    for (int64_t i = 0; i < nb && e == cudaSuccess; ++i) e = cudaGraphLaunch(b->graph, b->work);
    if ((st = bcheck(b, e, "attempt launch")) != LH_OK) return st;
    att += nb;
    // after the first batch: small, then doubling (the few instances that
    // redid steps finish within a few attempts)
    batch = (nb == first_batch && att == nb) ? 4 : (batch < 64 ? 2 * batch : 64);
  }
  cudaEventRecord(b->ev1, b->work);
  e = cudaEventSynchronize(b->ev1);
  if ((st = bcheck(b, e, "run sync")) != LH_OK) return st;
  if (wall_ms) cudaEventElapsedTime(wall_ms, b->ev0, b->ev1);
  if (launched) *launched = att;
  return LH_OK;
}

static void free_batch(lh_batch* b) {
  void* ptrs[] = {b->d_inst, b->d_order, b->d_ctl, b->v, b->e, b->x, b->vh, b->eh, b->xh,
                  b->vn, b->en, b->xn, b->vbar, b->rho0K, b->rho0Kinv, b->fac, b->F1E, b->FK, b->D,
                  b->srcE, b->vec, b->aux, b->qctr, b->ndone, b->d_snap_ov};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (b->ctl_host) cudaFreeHost(b->ctl_host);
  if (b->ndone_host) cudaFreeHost(b->ndone_host);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  if (b->ev0) cudaEventDestroy(b->ev0);
  if (b->ev1) cudaEventDestroy(b->ev1);
  if (b->own_work && b->work) cudaStreamDestroy(b->work);
}

template <typename T>
static cudaError_t balloc(T** p, size_t n) {
  return cudaMalloc((void**)p, (n > 0 ? n : 1) * sizeof(T));
}

}  // namespace lagh

extern "C" lh_status lh_batch_create(int32_t n, const lh_mesh_desc* meshes,
                                     const lh_disc_desc* disc, const lh_phys_desc* phys,
                                     int32_t precision, void* stream,
                                     const lh_batch_tuning* tuning, lh_batch** out) {
  if (!out) return LH_EINVAL;
  *out = nullptr;
  if (n < 1 || !meshes || !disc || !phys) return LH_EINVAL;
  if (precision != LH_FP64 && precision != LH_MIXED) return LH_EINVAL;
  lh_batch* b = new lh_batch();
  auto fail = [&](lh_status s, const std::string& m) {
    fprintf(stderr, "lh_batch_create: %s\n", m.c_str());
    free_batch(b);
    delete b;
    return s;
  };
  b->n = n;
  b->precision = precision;
  b->stream = (cudaStream_t)stream;
  b->inst.resize(n);
  b->phys.assign(phys, phys + n);
  b->off_v.assign(n + 1, 0);
  b->off_e.assign(n + 1, 0);
  b->off_el.assign(n + 1, 0);
  // ---- instances ----
  std::map<std::pair<int, int>, int64_t> fac_at;  // (elements, variant) -> table offset
  std::vector<double> fac;
  for (int i = 0; i < n; ++i) {
    Geom g;
    std::string why;
    lh_status gs = make_geom(&meshes[i], disc, &g, &why);
    if (gs != LH_OK) return fail(gs, "instance " + std::to_string(i) + ": " + why);
    if (i == 0) {
      b->dim = g.dim;
      b->k = g.k;
      build_basis(g.k, g.nq, g.dim, &b->basis);
    } else if (g.dim != b->dim) {
      return fail(LH_EINVAL, "every instance of a batch has the same dimension");
    }
    const lh_phys_desc& p = phys[i];
    if (!(p.gamma > 1.0)) return fail(LH_EINVAL, "gamma must exceed 1");
    if (p.problem < LH_SEDOV || p.problem > LH_TRIPLE_POINT) return fail(LH_EINVAL, "unknown problem");
    if (p.problem == LH_TRIPLE_POINT)
      return fail(LH_EUNSUPPORTED, "the batched form runs single-material problems (rho0 = 1)");
    if (p.integrator != LH_RK2AVG)
      return fail(LH_EUNSUPPORTED, "the batched form runs the RK2-average integrator");
    if (!(p.cg_rtol > 0.0) || p.cg_maxit < 1) return fail(LH_EINVAL, "bad CG settings");
    if (g.nv >= (int64_t(1) << 31))
      return fail(LH_EUNSUPPORTED, "an instance of the batched form holds fewer than 2^31 velocity unknowns");
    BInst& I = b->inst[i];
    memset(&I, 0, sizeof(I));
    I.g = g;
    I.ph.gamma = p.gamma;
    I.ph.cfl = p.cfl;
    I.ph.cfl_mu = p.cfl_mu;
    I.ph.q1 = p.q1;
    I.ph.q2 = p.q2;
    I.ph.visc = p.visc;
    I.ph.problem = p.problem;
    I.ph.source = (p.source && p.problem == LH_TAYLOR_GREEN && g.dim == 2) ? 1 : 0;
    set_phys_floats(I.ph);
    b->has_source |= I.ph.source;
    I.kc.beta1 = p.beta1;
    I.kc.beta2 = p.beta2;
    I.kc.gamma_dt = p.gamma_dt;
    I.rho0K = 1.0 * g.detJ0;  // rho0 = 1 in every problem
    I.scale = 1.0 / I.rho0K;
    I.ov = b->tot_v;
    I.oe = b->tot_e;
    I.oel = b->tot_el;
    b->tot_v += g.nv;
    b->tot_e += g.ne;
    b->tot_el += g.nelem;
    b->off_v[i + 1] = b->tot_v;
    b->off_e[i + 1] = b->tot_e;
    b->off_el[i + 1] = b->tot_el;
    b->max_nelem = std::max(b->max_nelem, g.nelem);
    b->max_nv = std::max(b->max_nv, g.nv);
    b->max_ne = std::max(b->max_ne, g.ne);
    b->max_nnodes = std::max(b->max_nnodes, g.nnodes);
    for (int d = 0; d < g.dim; ++d)
      for (int var = 0; var < 2; ++var) {
        auto key = std::make_pair(g.n[d], var);
        auto it = fac_at.find(key);
        if (it == fac_at.end()) {
          std::vector<double> L;
          banded_cholesky_1d(b->basis, g.k, g.n[d], var, L);
          // row r: d_r = 1 / L_rr, d_r L_{r,r-q}, d_r L_{r+q,r} (q = 1..k; zero
          // beyond the line)
          const int64_t off = (int64_t)fac.size();
          const int kk = g.k, rows = (int)(L.size() / (kk + 1));
          for (int r = 0; r < rows; ++r) {
            const double dr = 1.0 / L[(size_t)r * (kk + 1)];
            fac.push_back(dr);
            for (int q = 1; q <= kk; ++q) fac.push_back(dr * L[(size_t)r * (kk + 1) + q]);
            for (int q = 1; q <= kk; ++q)
              fac.push_back(r + q < rows ? dr * L[(size_t)(r + q) * (kk + 1) + q] : 0.0);
          }
          it = fac_at.emplace(key, off).first;
        }
        I.fac[d][var] = it->second;
      }
  }
  b->rtol = phys[0].cg_rtol;
  b->maxit = phys[0].cg_maxit;
  // largest first (ties by index): the queue order of the persistent kernels
  std::vector<int32_t> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t c) {
    return b->inst[a].g.nelem > b->inst[c].g.nelem;
  });
  // ---- device ----
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, dev);
  int optin = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return fail(LH_ECUDA, cudaGetErrorString(e));
  b->smem_optin = (size_t)optin - 2048;  // static shared memory of the kernels
  const int d = b->dim, k = b->k;
  int nd1 = 1, nd2 = 1, nqd = 1;
  for (int i = 0; i < d; ++i) { nd1 *= k + 1; nd2 *= k; nqd *= 2 * k; }
  auto al = [](int64_t v) { return (v + 31) & ~int64_t(31); };  // 256-byte slots
  b->s_f1e = al(b->max_nelem * d * nd1);
  b->s_fkd = precision == LH_MIXED ? al(b->max_nelem * d * nd1 * nd2)  // floats
                                   : al(b->max_nelem * d * d * nqd);  // doubles
  b->s_src = b->has_source ? al(b->max_ne) : 0;
  b->s_vec = al(5 * b->max_nv);
  // scratch for up to 4 CTAs per SM, within 8 GiB
  const int64_t per_slot = 8 * (b->s_f1e + b->s_src + b->s_vec) +
                           (precision == LH_MIXED ? 4 : 8) * b->s_fkd;
  int64_t slots = (int64_t)b->num_sms * 4;
  const int64_t budget = (int64_t)8 << 30;
  if (slots * per_slot > budget) slots = std::max<int64_t>(b->num_sms, budget / per_slot);
  b->slots = (int)slots;
  if (e == cudaSuccess) e = balloc(&b->d_inst, n);
  if (e == cudaSuccess) e = balloc(&b->d_order, n);
  if (e == cudaSuccess) e = balloc(&b->d_ctl, n);
  double** vv[] = {&b->v, &b->x, &b->vh, &b->xh, &b->vn, &b->xn, &b->vbar};
  for (double** p : vv)
    if (e == cudaSuccess) e = balloc(p, b->tot_v);
  double** ee[] = {&b->e, &b->eh, &b->en};
  for (double** p : ee)
    if (e == cudaSuccess) e = balloc(p, b->tot_e);
  if (e == cudaSuccess) e = balloc(&b->rho0K, b->tot_el);
  if (e == cudaSuccess) e = balloc(&b->rho0Kinv, b->tot_el);
  if (e == cudaSuccess) e = balloc(&b->fac, fac.size());
  if (e == cudaSuccess) e = balloc(&b->F1E, slots * b->s_f1e);
  if (precision == LH_MIXED) {
    if (e == cudaSuccess) e = balloc(&b->FK, slots * b->s_fkd);
  } else {
    if (e == cudaSuccess) e = balloc(&b->D, slots * b->s_fkd);
  }
  if (b->has_source && e == cudaSuccess) e = balloc(&b->srcE, slots * b->s_src);
  if (e == cudaSuccess) e = balloc(&b->vec, slots * b->s_vec);
  if (e == cudaSuccess) e = balloc(&b->aux, 2 * (size_t)n);
  if (e == cudaSuccess) e = balloc(&b->qctr, 8);
  if (e == cudaSuccess) e = balloc(&b->ndone, 1);
  if (e == cudaSuccess) e = balloc(&b->d_snap_ov, 3 * (size_t)n);
  if (e == cudaSuccess) e = cudaMemset(b->d_snap_ov, 0, sizeof(int64_t) * 3 * (size_t)n);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&b->ctl_host, sizeof(Ctl) * n);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&b->ndone_host, sizeof(int));
  if (e == cudaSuccess) e = cudaEventCreate(&b->ev0);
  if (e == cudaSuccess) e = cudaEventCreate(&b->ev1);
  if (e == cudaSuccess) {
    if (b->stream == nullptr) {
      e = cudaStreamCreateWithFlags(&b->work, cudaStreamNonBlocking);
      b->own_work = 1;
    } else {
      b->work = b->stream;
    }
  }
  if (e != cudaSuccess) {
    const bool oom = e == cudaErrorMemoryAllocation;
    cudaGetLastError();
    return fail(oom ? LH_ENOMEM : LH_ECUDA, cudaGetErrorString(e));
  }
  std::vector<double> r0(b->tot_el), r0i(b->tot_el);
  for (int i = 0; i < n; ++i)
    for (int64_t el = 0; el < b->inst[i].g.nelem; ++el) {
      r0[b->inst[i].oel + el] = b->inst[i].rho0K;
      r0i[b->inst[i].oel + el] = b->inst[i].scale;
    }
  std::vector<Ctl> c0(n);
  memset(c0.data(), 0, sizeof(Ctl) * n);
  e = cudaMemcpy(b->d_inst, b->inst.data(), sizeof(BInst) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_order, order.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_ctl, c0.data(), sizeof(Ctl) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->rho0K, r0.data(), sizeof(double) * b->tot_el, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->rho0Kinv, r0i.data(), sizeof(double) * b->tot_el, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !fac.empty())
    e = cudaMemcpy(b->fac, fac.data(), sizeof(double) * fac.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(b->qctr, 0, 8 * sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMemset(b->ndone, 0, sizeof(int));
  if (b->has_source && e == cudaSuccess) e = cudaMemset(b->srcE, 0, sizeof(double) * slots * b->s_src);
  if (e != cudaSuccess) return fail(LH_ECUDA, cudaGetErrorString(e));
  // ---- launch shape ----
  lh_batch_tuning t;
  memset(&t, 0, sizeof(t));
  if (tuning && tuning->threads > 0) {
    t = *tuning;
    b->tuned = 1;
  }
  lh_status st;
  if (b->tuned) {
    st = apply_tuning(b, t);
  } else {
    // default shape: the widest CTA built for this dimension whose shared
    // memory holds the largest instance's node lines (fewer staged if not)
    st = LH_EUNSUPPORTED;
    for (int ti = 2; ti >= 0 && st != LH_OK; --ti)
      for (int sl = 2; sl >= 0 && st != LH_OK; --sl) {
        t.threads = kThreadChoices[ti];
        t.ctas_per_sm = 0;
        t.smem_lines = sl;
        t.qpt = 1;
        st = apply_tuning(b, t);
      }
  }
  if (st != LH_OK) return fail(st, b->err);
  *out = b;
  return LH_OK;
}

extern "C" lh_status lh_batch_destroy(lh_batch* b) {
  if (!b) return LH_EINVAL;
  if (b->work) cudaStreamSynchronize(b->work);
  free_batch(b);
  delete b;
  return LH_OK;
}

extern "C" const char* lh_batch_last_error(const lh_batch* b) {
  return b ? b->err.c_str() : "null batch";
}

extern "C" lh_status lh_batch_layout(const lh_batch* b, int64_t* off_v, int64_t* off_e,
                                     lh_layout_info* info) {
  if (!b) return LH_EINVAL;
  for (int i = 0; i <= b->n; ++i) {
    if (off_v) off_v[i] = b->off_v[i];
    if (off_e) off_e[i] = b->off_e[i];
  }
  if (info)
    for (int i = 0; i < b->n; ++i) {
      const Geom& g = b->inst[i].g;
      lh_layout_info& L = info[i];
      memset(&L, 0, sizeof(L));
      L.nv = g.nv;
      L.ne = g.ne;
      L.nelem = g.nelem;
      L.nnodes = g.nnodes;
      L.dim = g.dim;
      L.order = g.k;
      L.nq = g.nq;
      int nd1 = 1, nd2 = 1, nqe = 1;
      for (int d = 0; d < g.dim; ++d) { nd1 *= g.k + 1; nd2 *= g.k; nqe *= g.nq; }
      L.nqp = g.nelem * nqe;
      L.ndof_h1 = nd1;
      L.ndof_l2 = nd2;
      L.nqe = nqe;
      for (int d = 0; d < 3; ++d) L.nodes_per_dim[d] = g.nn[d];
      L.precision = b->precision;
      int64_t ness = 0;
      for (int c = 0; c < g.dim; ++c) ness += 2 * (g.nnodes / g.nn[c]);
      L.n_essential = ness;
    }
  return LH_OK;
}

extern "C" lh_status lh_batch_tuning_get(const lh_batch* b, lh_batch_tuning* t) {
  if (!b || !t) return LH_EINVAL;
  *t = b->tune;
  return LH_OK;
}

static lh_status reset_ctl(lh_batch* b, const double* t, const double* dt) {
  std::vector<Ctl> c0(b->n);
  memset(c0.data(), 0, sizeof(Ctl) * b->n);
  for (int i = 0; i < b->n; ++i) {
    c0[i].t = t ? t[i] : 0.0;
    c0[i].dt = dt ? dt[i] : 0.0;
  }
  cudaError_t e = cudaMemcpyAsync(b->d_ctl, c0.data(), sizeof(Ctl) * b->n, cudaMemcpyHostToDevice,
                                  b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  return bcheck(b, e, "control blocks");
}

extern "C" lh_status lh_batch_init_state(lh_batch* b) {
  if (!b) return LH_EINVAL;
  std::vector<double> V(b->tot_v), E(b->tot_e), X(b->tot_v);
  for (int i = 0; i < b->n; ++i) {
    std::vector<double> v, e, x;
    initial_state(b->inst[i].g, b->phys[i], v, e, x);
    std::copy(v.begin(), v.end(), V.begin() + b->off_v[i]);
    std::copy(x.begin(), x.end(), X.begin() + b->off_v[i]);
    std::copy(e.begin(), e.end(), E.begin() + b->off_e[i]);
  }
  cudaError_t e = cudaMemcpyAsync(b->v, V.data(), 8 * b->tot_v, cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->x, X.data(), 8 * b->tot_v, cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->e, E.data(), 8 * b->tot_e, cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  lh_status st = bcheck(b, e, "init_state upload");
  if (st != LH_OK) return st;
  return reset_ctl(b, nullptr, nullptr);
}

extern "C" lh_status lh_batch_set_state(lh_batch* b, const double* v, const double* e,
                                        const double* x, const double* t, const double* dt) {
  if (!b || !v || !e || !x) return LH_EINVAL;
  cudaError_t err = cudaMemcpyAsync(b->v, v, 8 * b->tot_v, cudaMemcpyDefault, b->stream);
  if (err == cudaSuccess) err = cudaMemcpyAsync(b->x, x, 8 * b->tot_v, cudaMemcpyDefault, b->stream);
  if (err == cudaSuccess) err = cudaMemcpyAsync(b->e, e, 8 * b->tot_e, cudaMemcpyDefault, b->stream);
  if (err == cudaSuccess) err = cudaStreamSynchronize(b->stream);
  lh_status st = bcheck(b, err, "set_state");
  if (st != LH_OK) return st;
  return reset_ctl(b, t, dt);
}

extern "C" lh_status lh_batch_get_state(lh_batch* b, double* v, double* e, double* x) {
  if (!b) return LH_EINVAL;
  cudaError_t err = cudaSuccess;
  if (v) err = cudaMemcpyAsync(v, b->v, 8 * b->tot_v, cudaMemcpyDefault, b->stream);
  if (err == cudaSuccess && x) err = cudaMemcpyAsync(x, b->x, 8 * b->tot_v, cudaMemcpyDefault, b->stream);
  if (err == cudaSuccess && e) err = cudaMemcpyAsync(e, b->e, 8 * b->tot_e, cudaMemcpyDefault, b->stream);
  if (err == cudaSuccess) err = cudaStreamSynchronize(b->stream);
  return bcheck(b, err, "get_state");
}

extern "C" lh_status lh_batch_query(lh_batch* b, double* t, double* dt, int64_t* steps,
                                    int64_t* rejects, int64_t* cg_iters, int32_t* status) {
  if (!b) return LH_EINVAL;
  lh_status st;
  if ((st = bcheck(b, join(b, true), "stream join")) != LH_OK) return st;
  if ((st = read_ctl(b)) != LH_OK) return st;
  for (int i = 0; i < b->n; ++i) {
    const Ctl& c = b->ctl_host[i];
    if (t) t[i] = c.t;
    if (dt) dt[i] = c.dt;
    if (steps) steps[i] = c.steps;
    if (rejects) rejects[i] = c.rejects;
    if (cg_iters) cg_iters[i] = c.cg_iters;
    if (status) {
      lh_status s = LH_OK;
      if (c.status & kDevNonFinite) s = LH_ENONFINITE;
      else if (c.status & kDevCG) s = LH_ECG;
      else if (c.status & kDevDtMin) s = LH_EDTMIN;
      status[i] = s;
    }
  }
  return LH_OK;
}

static lh_status batch_run(lh_batch* b, double t_final, int64_t max_steps, int fixed,
                           const double* dt_fixed, lh_batch_stats* stats) {
  lh_status st;
  if ((st = bcheck(b, join(b, true), "stream join")) != LH_OK) return st;
  if ((st = begin_run(b, t_final, max_steps, fixed, dt_fixed)) != LH_OK) return st;
  float ms = 0.f;
  int64_t launched = 0;
  // every attempt of an unfinished instance is accepted, rejected or ends it;
  // 60 rejections in a row take dt below any dt_min fraction above 1e-5
  const int64_t max_att = fixed ? 1 : (max_steps > INT64_MAX / 64 ? INT64_MAX : 61 * (max_steps + 1));
  const int64_t first = fixed ? 1 : (max_steps < 63 ? max_steps + 1 : 64);
  if ((st = run_loop(b, max_att, first, &ms, &launched)) != LH_OK) return st;
  if ((st = read_ctl(b)) != LH_OK) return st;
  if ((st = bcheck(b, join(b, false), "stream join")) != LH_OK) return st;
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    for (int i = 0; i < b->n; ++i) {
      const Ctl& c = b->ctl_host[i];
      stats->steps += c.steps;
      stats->rejects += c.rejects;
      stats->cg_iters += c.cg_iters;
      stats->attempts += c.attempts;
      stats->instances_done += c.done ? 1 : 0;
      const BInst& I = b->inst[i];
      stats->dof_updates += (2 * I.g.nv + I.g.ne) * c.steps;
    }
    stats->graph_launches = launched;
    stats->wall_ms = ms;
  }
  return instance_status(b);
}

extern "C" lh_status lh_batch_snapshots(lh_batch* b, int32_t nsel, const int32_t* ids,
                                        int64_t cap, double* Sv, double* Se, double* Sx) {
  if (!b || nsel < 0 || nsel > b->n || cap < 0) return LH_EINVAL;
  if (nsel > 0 && (!ids || !Sv || !Se || !Sx || cap < 1)) return LH_EINVAL;
  lh_status st;
  if ((st = bcheck(b, join(b, true), "stream join")) != LH_OK) return st;
  std::vector<int64_t> h(3 * (size_t)b->n, 0);
  for (int i = 0; i < b->n; ++i) h[i] = h[b->n + i] = -1;
  int64_t ov = 0, oe = 0;
  for (int s = 0; s < nsel; ++s) {
    const int i = ids[s];
    if (i < 0 || i >= b->n || (s > 0 && i <= ids[s - 1]))
      return bset_error(b, LH_EINVAL, "snapshot ids must be ascending instance indices");
    h[i] = ov;
    h[b->n + i] = oe;
    ov += cap * b->inst[i].g.nv;
    oe += cap * b->inst[i].g.ne;
  }
  cudaError_t e = cudaMemcpyAsync(b->d_snap_ov, h.data(), sizeof(int64_t) * 3 * b->n, cudaMemcpyHostToDevice,
                      b->work);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->work);
  if ((st = bcheck(b, e, "snapshot tables")) != LH_OK) return st;
  b->Sv = Sv;
  b->Se = Se;
  b->Sx = Sx;
  b->snap_cap = cap;
  b->snap_on = nsel > 0;
  if (b->graph) {  // the attempt graph holds the kernel arguments: rebuild it
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  return bcheck(b, join(b, false), "stream join");
}

extern "C" lh_status lh_batch_snapshot_count(lh_batch* b, int64_t* counts) {
  if (!b || !counts) return LH_EINVAL;
  lh_status st;
  if ((st = bcheck(b, join(b, true), "stream join")) != LH_OK) return st;
  cudaError_t e = cudaMemcpyAsync(counts, b->d_snap_ov + 2 * b->n, sizeof(int64_t) * b->n,
                                  cudaMemcpyDeviceToHost, b->work);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->work);
  return bcheck(b, e, "snapshot counts");
}

extern "C" lh_status lh_batch_run_to(lh_batch* b, double t_final, int64_t max_steps,
                                     lh_batch_stats* stats) {
  if (!b || !(t_final >= 0.0) || max_steps < 0) return LH_EINVAL;
  return batch_run(b, t_final, max_steps, 0, nullptr, stats);
}

extern "C" lh_status lh_batch_step_fixed(lh_batch* b, const double* dt, lh_batch_stats* stats) {
  if (!b || !dt) return LH_EINVAL;
  for (int i = 0; i < b->n; ++i)
    if (!(dt[i] > 0.0)) return LH_EINVAL;
  return batch_run(b, 1e300, INT64_MAX / 2, 1, dt, stats);
}

extern "C" lh_status lh_batch_total_energy(lh_batch* b, double* energy) {
  if (!b || !energy) return LH_EINVAL;
  BatchArgs a = bargs(b);
  a.out = b->aux;
  lh_status st;
  if ((st = launch_aux(b, b->ops.energy, b->ops.energy_bytes, a, nullptr, b->stream)) != LH_OK)
    return st;
  cudaError_t e = cudaMemcpyAsync(energy, b->aux, sizeof(double) * b->n, cudaMemcpyDeviceToHost,
                                  b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  return bcheck(b, e, "total energy");
}

extern "C" lh_status lh_batch_force_sampled(lh_batch* b, const int64_t* list_off,
                                            const int32_t* elem_ids, const double* v,
                                            const double* e, const double* x,
                                            const double* vtest, double* F1_local,
                                            double* FTv_local, double* dt_est) {
  if (!b || !list_off || !F1_local) return LH_EINVAL;
  BatchArgs a = bargs(b);
  if (v) a.v = const_cast<double*>(v);
  if (e) a.e = const_cast<double*>(e);
  if (x) a.x = const_cast<double*>(x);
  a.list_off = list_off;
  a.list = elem_ids;
  a.vtest = vtest;
  a.out = F1_local;
  a.out2 = vtest ? FTv_local : nullptr;
  unsigned long long* est = reinterpret_cast<unsigned long long*>(b->aux);
  lh_status st = launch_aux(b, b->ops.sampled, b->stage_smem, a, &est, b->stream);
  if (st != LH_OK) return st;
  if (dt_est) {
    cudaError_t err = cudaMemcpyAsync(dt_est, b->aux, sizeof(double) * b->n,
                                      cudaMemcpyDeviceToHost, b->stream);
    if (err == cudaSuccess) err = cudaStreamSynchronize(b->stream);
    if ((st = bcheck(b, err, "sampled estimates")) != LH_OK) return st;
  }
  return LH_OK;
}

// Autotuner: times the stage kernel of the current states for every launch
// shape that fits (threads per CTA, so elements per force tile and per mass
// tile; CTAs per SM; node lines staged in shared memory or not) and keeps the
// fastest.  The states are not changed: stage 0 writes only the half-step
// arrays, and the control blocks are restored.
extern "C" lh_status lh_batch_autotune(lh_batch* b, int32_t reps, lh_batch_tuning* chosen) {
  if (!b) return LH_EINVAL;
  if (reps < 1) reps = 2;
  lh_status st;
  if ((st = bcheck(b, join(b, true), "stream join")) != LH_OK) return st;
  if ((st = read_ctl(b)) != LH_OK) return st;
  std::vector<Ctl> saved(b->ctl_host, b->ctl_host + b->n);
  const lh_batch_tuning keep = b->tune;
  // a run start gives every instance a step size (estimate) and clears done
  if ((st = begin_run(b, 1e300, INT64_MAX / 2, 0, nullptr)) != LH_OK) return st;
  float best = 1e30f;
  lh_batch_tuning best_t = keep;
  for (int qpt = 1; qpt <= 2; ++qpt)
  for (int ti = 0; ti < 3; ++ti)
    for (int sl = 2; sl >= 0; --sl)
      for (int cps = 1; cps <= 4; ++cps) {
        lh_batch_tuning t;
        memset(&t, 0, sizeof(t));
        t.threads = kThreadChoices[ti];
        t.smem_lines = sl;
        t.ctas_per_sm = cps;
        t.qpt = qpt;
        if (apply_tuning(b, t) != LH_OK) continue;
        if (b->tune.ctas_per_sm != cps) continue;  // more than fit
        if ((int64_t)b->num_sms * cps > b->slots) continue;
        cudaError_t e = launch_stage(b, 0, b->work);  // warm-up
        if (e == cudaSuccess) e = cudaEventRecord(b->ev0, b->work);
        for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch_stage(b, 0, b->work);
        if (e == cudaSuccess) e = cudaEventRecord(b->ev1, b->work);
        if (e == cudaSuccess) e = cudaEventSynchronize(b->ev1);
        if ((st = bcheck(b, e, "autotune")) != LH_OK) return st;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, b->ev0, b->ev1);
        if (ms < best) {
          best = ms;
          best_t = b->tune;
        }
      }
  b->err.clear();
  cudaError_t e = cudaMemcpyAsync(b->d_ctl, saved.data(), sizeof(Ctl) * b->n,
                                  cudaMemcpyHostToDevice, b->work);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->work);
  if ((st = bcheck(b, e, "autotune restore")) != LH_OK) return st;
  if ((st = apply_tuning(b, best_t)) != LH_OK) return st;
  b->tuned = 1;
  if (chosen) *chosen = b->tune;
  return bcheck(b, join(b, false), "stream join");
}
