// Preconditioned CG for the kinematic mass matrix (momentum equation of
// eq:fom: M_V a = -F.1 on the non-essential components).
//
// The solve is a chain of ordinary kernels, one per phase, so it can live in
// the step's CUDA graph: the iterations are a graph WHILE node whose condition
// the update kernel clears once ||r|| <= rtol ||b||.  Every reduction is
// deterministic: each block writes its partial sum, the last block to finish
// (ticket counter) adds the partials in block order and publishes the scalar.
//
// Preconditioners:
//  - tensor product: with rho0|J0| the same in every element, M_s is
//    rho0|J0| G_x (x) G_y [(x) G_z] with G_d the assembled 1D reference mass
//    matrices; its inverse is applied by banded Cholesky solves along every
//    node line, one direction per kernel.  This is the exact inverse, so the
//    CG stops after one iteration;
//  - Jacobi: the inverse assembled diagonal.
#include "mass_ops.cuh"

namespace lagh {

constexpr int kLineThreads = 32;
constexpr int kNodeThreads = 256;
enum { kTicketPass0 = 0, kTicketPassL = 1, kTicketA = 2, kTicketB = 3, kTicketJ = 4 };

struct CgArgs {
  Geom g;
  double M1[(kMaxOrder + 1) * (kMaxOrder + 1)];
  TensorPC tpc;
  const float* lfac;
  const double* rhs;
  double *x, *r, *z, *p, *Ap, *ApE;
  const double* dinv;
  const double* rho0K;
  double* part;          // partial sums [5][kMaxPartials]
  CgDev* cg;
  Ctl* ctl;              // reports and error bits
  const Ctl* gate;       // if set and done, every kernel returns
  double rtol;
  int maxit;
  int has_cond;
  cudaGraphConditionalHandle cond;
};

__device__ __forceinline__ bool gated(const CgArgs& a) {
  return (a.gate != nullptr && a.gate->done) || a.cg->done;
}

// Block partial -> last block adds all partials in block order.  Returns true
// in every thread of the last block; *total is valid there.
__device__ __forceinline__ bool reduce_last(double v, double* part, unsigned int* ticket,
                                            double* total) {
  __shared__ double sh[32];
  __shared__ bool last;
  double s = block_sum(v, sh);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = s;
    __threadfence();
    unsigned int t = atomicAdd(ticket, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return false;
  if (threadIdx.x == 0) {
    __threadfence();
    double acc = 0.0;
    for (unsigned int i = 0; i < gridDim.x; ++i) acc += __ldcg(&part[i]);
    *total = acc;
    *ticket = 0u;
  }
  __syncthreads();
  return true;
}

// Block partial only (the caller's last block reads it back).
__device__ __forceinline__ void write_partial(double v, double* part) {
  __shared__ double sh[32];
  double s = block_sum(v, sh);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = s;
    __threadfence();
  }
}

__device__ __forceinline__ double sum_partials(const double* part) {
  double acc = 0.0;
  for (unsigned int i = 0; i < gridDim.x; ++i) acc += __ldcg(&part[i]);
  return acc;
}

__device__ __forceinline__ void report(const CgArgs& a, bool conv, double rr) {
  CgDev* cg = a.cg;
  a.ctl->cg_last_iters = cg->it;
  a.ctl->cg_last_relres = cg->bb > 0.0 ? sqrt(rr / cg->bb) : 0.0;
  a.ctl->cg_iters += cg->it;
  if (!conv) atomicOr(&a.ctl->status, kDevCG);
}

// ---------------------------------------------------- tensor line passes --

// One warp owns 32 node lines of one direction (consecutive line numbers): it
// stages them in shared memory with coalesced loads, each lane runs the banded
// forward/backward substitution of its line from shared memory in FP32, and
// the warp writes the lines back with coalesced stores.
//
// mode: 0 = first pass of the initial preconditioning (reads rhs, writes r = b
// on free components and x = 0, sums b.b), 1 = first pass inside the loop
// (reads r), 2 = later pass (in place on z).  last: the pass along the last
// direction (sums r.z; init also writes p = z).
template <int DIM, int K>
__global__ void __launch_bounds__(kLineThreads) cg_pass_kernel(const CgArgs a, int d, int mode,
                                                              int last, int init) {
  if (init ? (a.gate != nullptr && a.gate->done) : gated(a)) return;
  if (mode == 0 && blockIdx.x == 0 && threadIdx.x == 0) {  // a new solve
    a.cg->done = 0;
    a.cg->it = 0;
  }
  extern __shared__ float lines[];  // [32][ld], ld odd: conflict-free lane rows
  const Geom& g = a.g;
  const int nd = g.nn[d];
  const int ld = nd | 1;
  const int64_t nlines = g.nnodes / nd;
  const int64_t stride = d == 0 ? 1 : (d == 1 ? (int64_t)g.nn[0] : (int64_t)g.nn[0] * g.nn[1]);
  const int lane = threadIdx.x;
  const int64_t task = (int64_t)blockIdx.x * 32 + lane;
  const bool active = task < DIM * nlines;
  int c = 0;
  int I[3] = {0, 0, 0};
  int64_t base = 0;
  bool wall_line = true;
  if (active) {
    c = (int)(task / nlines);
    const int64_t line = task - (int64_t)c * nlines;
    if (d == 0) { I[1] = (int)(line % g.nn[1]); I[2] = (int)(line / g.nn[1]); }
    else if (d == 1) { I[0] = (int)(line % g.nn[0]); I[2] = (int)(line / g.nn[0]); }
    else { I[0] = (int)(line % g.nn[0]); I[1] = (int)(line / g.nn[0]); }
    base = (int64_t)c * g.nnodes + node_index(g, I[0], I[1], I[2]);
    wall_line = (c != d) && (I[c] == 0 || I[c] == g.nn[c] - 1);
  }
  const double* src = mode == 0 ? a.rhs : (mode == 1 ? a.r : a.z);
  float* my = lines + lane * ld;
  double l_bb = 0.0, l_rz = 0.0;
  const float scl = (mode == 2) ? 1.0f : (float)a.tpc.scale;

  // ---- load: entry i of the line of lane l ----
  auto load_entry = [&](int l, int64_t bl, int cl, bool wl, int i) {
    const int64_t k = bl + i * stride;
    const bool ess = wl || (cl == d && (i == 0 || i == nd - 1));
    double v = ess ? 0.0 : src[k];
    if (mode == 0) {
      a.r[k] = v;
      a.x[k] = 0.0;
      l_bb += v * v;
    }
    lines[l * ld + i] = (float)v * scl;
  };
  if (d == 0) {
    // lines are contiguous rows: the warp loads row after row
    for (int l = 0; l < 32; ++l) {
      const int64_t bl = __shfl_sync(0xffffffffu, base, l);
      const int cl = __shfl_sync(0xffffffffu, c, l);
      const int wl = __shfl_sync(0xffffffffu, (int)wall_line, l);
      const int al = __shfl_sync(0xffffffffu, (int)active, l);
      if (!al) continue;
      for (int i = lane; i < nd; i += 32) load_entry(l, bl, cl, wl != 0, i);
    }
  } else if (active) {
    // neighbouring lanes hold neighbouring lines: every load is coalesced
    for (int i = 0; i < nd; ++i) load_entry(lane, base, c, wall_line, i);
  }
  __syncwarp();

  // ---- banded Cholesky solve of this lane's line (FP32, shared memory) ----
  if (active && !wall_line) {
    const int var = (c == d) ? 1 : 0;
    const int N = nd - 2 * var;
    const float* L = a.lfac + a.tpc.off[d][var];  // L[i][0] holds 1 / L_ii
    float* z = my + var;
    float win[K];
#pragma unroll
    for (int m = 0; m < K; ++m) win[m] = 0.0f;
    for (int i = 0; i < N; ++i) {
      const float* Li = L + i * (K + 1);
      float zz = z[i];
#pragma unroll
      for (int m = 1; m <= K; ++m) zz -= Li[m] * win[m - 1];
      const float y = zz * Li[0];
#pragma unroll
      for (int m = K - 1; m > 0; --m) win[m] = win[m - 1];
      win[0] = y;
      z[i] = y;
    }
#pragma unroll
    for (int m = 0; m < K; ++m) win[m] = 0.0f;
    for (int i = N - 1; i >= 0; --i) {
      float yy = z[i];
#pragma unroll
      for (int m = 1; m <= K; ++m)
        if (i + m < N) yy -= L[(i + m) * (K + 1) + m] * win[m - 1];
      const float xv = yy * L[i * (K + 1)];
#pragma unroll
      for (int m = K - 1; m > 0; --m) win[m] = win[m - 1];
      win[0] = xv;
      z[i] = xv;
    }
    if (var) {
      my[0] = 0.0f;
      my[nd - 1] = 0.0f;
    }
  }
  __syncwarp();

  // ---- store z (and p = z, r.z on the last pass) ----
  auto store_entry = [&](int l, int64_t bl, int i) {
    const int64_t k = bl + i * stride;
    const double zv = (double)lines[l * ld + i];
    a.z[k] = zv;
    if (last) {
      l_rz += a.r[k] * zv;
      if (init) a.p[k] = zv;
    }
  };
  if (d == 0) {
    for (int l = 0; l < 32; ++l) {
      const int64_t bl = __shfl_sync(0xffffffffu, base, l);
      const int al = __shfl_sync(0xffffffffu, (int)active, l);
      if (!al) continue;
      for (int i = lane; i < nd; i += 32) store_entry(l, bl, i);
    }
  } else if (active) {
    for (int i = 0; i < nd; ++i) store_entry(lane, base, i);
  }

  double tot;
  if (mode == 0) {
    if (reduce_last(l_bb, a.part, &a.cg->ticket[kTicketPass0], &tot) && threadIdx.x == 0)
      a.cg->bb = tot;
  }
  if (last) {
    if (reduce_last(l_rz, a.part + kMaxPartials, &a.cg->ticket[kTicketPassL], &tot) &&
        threadIdx.x == 0) {
      CgDev* cg = a.cg;
      if (init) {
        cg->rz = tot;
        cg->it = 0;
        if (!(cg->bb > 0.0)) {  // zero right-hand side: x = 0 is the solution
          cg->done = 1;
          report(a, true, 0.0);
        }
      } else {
        cg->beta = tot / cg->rz;
        cg->rz = tot;
      }
    }
  }
}

// ------------------------------------------------------- Jacobi init ----

template <int DIM, int K>
__global__ void __launch_bounds__(kNodeThreads) cg_jacobi_init_kernel(const CgArgs a) {
  if (a.gate != nullptr && a.gate->done) return;
  const Geom& g = a.g;
  double l_bb = 0.0, l_rz = 0.0;
  for (int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; node < g.nnodes;
       node += (int64_t)gridDim.x * blockDim.x) {
    int I[3];
    node_ijk(g, node, I);
    const double di = a.dinv[node];
    for (int c = 0; c < DIM; ++c) {
      const int64_t k = c * g.nnodes + node;
      const double bv = essential(g, I, c) ? 0.0 : a.rhs[k];
      a.r[k] = bv;
      a.x[k] = 0.0;
      const double zv = bv * di;
      a.z[k] = zv;
      a.p[k] = zv;
      l_bb += bv * bv;
      l_rz += bv * zv;
    }
  }
  write_partial(l_bb, a.part);
  double rz;
  if (reduce_last(l_rz, a.part + kMaxPartials, &a.cg->ticket[kTicketJ], &rz) &&
      threadIdx.x == 0) {
    CgDev* cg = a.cg;
    cg->bb = sum_partials(a.part);
    cg->rz = rz;
    cg->it = 0;
    if (!(cg->bb > 0.0)) {
      cg->done = 1;
      report(a, true, 0.0);
    }
  }
}

// ------------------------------------------------------ loop kernels ----

template <int DIM, int K>
__global__ void __launch_bounds__(256) cg_elem_kernel(const CgArgs a) {
  using L = ML<DIM, K>;
  constexpr int P = L::P, ND1 = L::ND1, EPB = L::EPB;
  if (gated(a)) return;
  __shared__ double M1s[P * P];
  __shared__ double u[EPB * DIM * ND1], t[EPB * DIM * ND1], y[EPB * DIM * ND1];
  (void)M1s;
  const Geom& g = a.g;
  for (int i = threadIdx.x; i < P * P; i += blockDim.x) M1s[i] = a.M1[(i / P) * (kMaxOrder + 1) + i % P];
  const int64_t el0 = (int64_t)blockIdx.x * EPB;
  const int nel = (int)((g.nelem - el0) < EPB ? (g.nelem - el0) : EPB);
  mass_elements<DIM, K>(g, M1s, a.p, a.rho0K, a.ApE, el0, nel, u, t, y);
}

template <int DIM, int K>
__global__ void __launch_bounds__(kNodeThreads) cg_gather_kernel(const CgArgs a) {
  if (gated(a)) return;
  const Geom& g = a.g;
  double l = 0.0;
  for (int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; node < g.nnodes;
       node += (int64_t)gridDim.x * blockDim.x) {
    int I[3];
    node_ijk(g, node, I);
    for (int c = 0; c < DIM; ++c) {
      const int64_t k = c * g.nnodes + node;
      const double ap = essential(g, I, c) ? 0.0 : gather_node<DIM, K>(g, a.ApE, I, c);
      a.Ap[k] = ap;
      l += a.p[k] * ap;
    }
  }
  double tot;
  if (reduce_last(l, a.part + 2 * kMaxPartials, &a.cg->ticket[kTicketA], &tot) && threadIdx.x == 0)
    a.cg->alpha = a.cg->rz / tot;
}

// x += alpha p, r -= alpha Ap; convergence test; ends the WHILE loop.
template <int DIM, int K>
__global__ void __launch_bounds__(kNodeThreads) cg_update_kernel(const CgArgs a, int jacobi) {
  if (gated(a)) {
    if (blockIdx.x == 0 && threadIdx.x == 0 && a.has_cond) cudaGraphSetConditional(a.cond, 0);
    return;
  }
  const Geom& g = a.g;
  const double alpha = a.cg->alpha;
  double l_rr = 0.0, l_rz = 0.0;
  for (int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; node < g.nnodes;
       node += (int64_t)gridDim.x * blockDim.x) {
    const double di = a.dinv[node];
    for (int c = 0; c < DIM; ++c) {
      const int64_t k = c * g.nnodes + node;
      a.x[k] += alpha * a.p[k];
      const double rv = a.r[k] - alpha * a.Ap[k];
      a.r[k] = rv;
      l_rr += rv * rv;
      if (jacobi) {
        const double zv = rv * di;
        a.z[k] = zv;
        l_rz += rv * zv;
      }
    }
  }
  if (jacobi) write_partial(l_rz, a.part + 3 * kMaxPartials);
  double rr;
  if (reduce_last(l_rr, a.part + 4 * kMaxPartials, &a.cg->ticket[kTicketB], &rr) &&
      threadIdx.x == 0) {
    CgDev* cg = a.cg;
    // every block wrote its r.z partial before taking its rr ticket
    const double rz_new = jacobi ? sum_partials(a.part + 3 * kMaxPartials) : 0.0;
    cg->it += 1;
    const bool conv = rr <= a.rtol * a.rtol * cg->bb;
    const bool bad = !(rr == rr);
    if (conv || bad || cg->it >= a.maxit) {
      cg->done = 1;
      report(a, conv, rr);
      if (a.has_cond) cudaGraphSetConditional(a.cond, 0);
    } else if (jacobi) {
      cg->beta = rz_new / cg->rz;
      cg->rz = rz_new;
    }
  }
}

template <int DIM, int K>
__global__ void __launch_bounds__(kNodeThreads) cg_pupdate_kernel(const CgArgs a) {
  if (gated(a)) return;
  const double beta = a.cg->beta;
  const int64_t n = (int64_t)DIM * a.g.nnodes;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    a.p[k] = a.z[k] + beta * a.p[k];
}

__global__ void cg_reset_kernel(CgDev* cg, const Ctl* gate) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    cg->done = 0;
    cg->it = 0;
  }
}

// ---------------------------------------------------------- launchers ----

static int node_grid(const lh_ctx* c) {
  int64_t b = (c->g.nnodes + kNodeThreads - 1) / kNodeThreads;
  int64_t cap = (int64_t)c->num_sms * 4;
  if (cap > kMaxPartials) cap = kMaxPartials;
  return (int)(b < cap ? (b > 0 ? b : 1) : cap);
}

static CgArgs make_args(const lh_ctx* c, const double* rhs, double* out, const Ctl* gate) {
  CgArgs a;
  a.g = c->g;
  for (int i = 0; i <= kMaxOrder; ++i)
    for (int j = 0; j <= kMaxOrder; ++j) a.M1[i * (kMaxOrder + 1) + j] = c->basis.M1[i][j];
  a.tpc = c->tpc;
  a.lfac = c->a.lfac;
  a.rhs = rhs;
  a.x = out;
  a.r = c->a.r;
  a.z = c->a.z;
  a.p = c->a.p;
  a.Ap = c->a.Ap;
  a.ApE = c->a.ApE;
  a.dinv = c->a.dinv;
  a.rho0K = c->a.rho0K;
  a.part = c->a.partials;
  a.cg = c->a.cg;
  a.ctl = c->a.ctl;
  a.gate = gate;
  a.rtol = c->cg_rtol;
  a.maxit = c->cg_maxit;
  a.has_cond = 0;
  a.cond = 0;
  return a;
}

template <int DIM, int K>
static cudaError_t precond_passes(const lh_ctx* c, const CgArgs& a, bool init, cudaStream_t s) {
  for (int d = 0; d < DIM; ++d) {
    const int64_t tasks = (int64_t)DIM * (c->g.nnodes / c->g.nn[d]);
    const int blocks = (int)((tasks + kLineThreads - 1) / kLineThreads);
    const int mode = d == 0 ? (init ? 0 : 1) : 2;
    const size_t smem = (size_t)32 * (c->g.nn[d] | 1) * sizeof(float);
    cg_pass_kernel<DIM, K><<<blocks, kLineThreads, smem, s>>>(a, d, mode, d == DIM - 1,
                                                              init ? 1 : 0);
  }
  return cudaGetLastError();
}

template <int DIM, int K>
static cudaError_t cg_init_dk(const lh_ctx* c, const CgArgs& a, cudaStream_t s) {
  if (c->tpc.enabled) return precond_passes<DIM, K>(c, a, true, s);
  cg_reset_kernel<<<1, 32, 0, s>>>(c->a.cg, a.gate);
  cg_jacobi_init_kernel<DIM, K><<<node_grid(c), kNodeThreads, 0, s>>>(a);
  return cudaGetLastError();
}

template <int DIM, int K>
static cudaError_t cg_body_dk(const lh_ctx* c, const CgArgs& a, cudaStream_t s) {
  using L = ML<DIM, K>;
  const int eblocks = (int)((c->g.nelem + L::EPB - 1) / L::EPB);
  cg_elem_kernel<DIM, K><<<eblocks, 256, 0, s>>>(a);
  cg_gather_kernel<DIM, K><<<node_grid(c), kNodeThreads, 0, s>>>(a);
  cg_update_kernel<DIM, K><<<node_grid(c), kNodeThreads, 0, s>>>(a, c->tpc.enabled ? 0 : 1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (c->tpc.enabled) {
    if ((e = precond_passes<DIM, K>(c, a, false, s)) != cudaSuccess) return e;
  }
  cg_pupdate_kernel<DIM, K><<<node_grid(c), kNodeThreads, 0, s>>>(a);
  return cudaGetLastError();
}

#define LAGH_DISPATCH_CG(FN, ...)                                           \
  do {                                                                      \
    const int D_ = c->g.dim, K_ = c->g.k;                                   \
    if (D_ == 2 && K_ == 1) return FN<2, 1>(__VA_ARGS__);                   \
    if (D_ == 2 && K_ == 2) return FN<2, 2>(__VA_ARGS__);                   \
    if (D_ == 2 && K_ == 3) return FN<2, 3>(__VA_ARGS__);                   \
    if (D_ == 3 && K_ == 1) return FN<3, 1>(__VA_ARGS__);                   \
    if (D_ == 3 && K_ == 2) return FN<3, 2>(__VA_ARGS__);                   \
    return cudaErrorInvalidValue;                                           \
  } while (0)

static cudaError_t cg_init(const lh_ctx* c, const CgArgs& a, cudaStream_t s) {
  LAGH_DISPATCH_CG(cg_init_dk, c, a, s);
}

static cudaError_t cg_body(const lh_ctx* c, const CgArgs& a, cudaStream_t s) {
  LAGH_DISPATCH_CG(cg_body_dk, c, a, s);
}

template <int DIM, int K>
static cudaError_t cg_prepare_dk(const lh_ctx* c) {
  int most = 0;
  for (int d = 0; d < DIM; ++d) most = c->g.nn[d] > most ? c->g.nn[d] : most;
  const int bytes = 32 * (most | 1) * (int)sizeof(float);
  return cudaFuncSetAttribute(cg_pass_kernel<DIM, K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              bytes);
}

// Shared memory of the line passes, set before any stream capture.
cudaError_t cg_prepare(const lh_ctx* c) { LAGH_DISPATCH_CG(cg_prepare_dk, c); }

// Eager solve (API): the body is launched in batches and the host polls the
// done flag between batches.
cudaError_t cg_solve_eager(const lh_ctx* c, const double* rhs, double* out, cudaStream_t s,
                           int* done_host) {
  CgArgs a = make_args(c, rhs, out, nullptr);
  cudaError_t e = cg_init(c, a, s);
  if (e != cudaSuccess) return e;
  for (int it = 0; it < c->cg_maxit + 1; it += 8) {
    for (int j = 0; j < 8; ++j)
      if ((e = cg_body(c, a, s)) != cudaSuccess) return e;
    e = cudaMemcpyAsync(done_host, &c->a.cg->done, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    if (*done_host) break;
  }
  return cudaSuccess;
}

// Inside a stream capture on s: the init kernels, then a WHILE conditional
// node whose body (captured on `side`) is one CG iteration.
cudaError_t cg_solve_capture(const lh_ctx* c, const double* rhs, double* out, const Ctl* gate,
                             cudaStream_t s, cudaStream_t side) {
  CgArgs a = make_args(c, rhs, out, gate);
  cudaError_t e = cg_init(c, a, s);
  if (e != cudaSuccess) return e;
  cudaStreamCaptureStatus cs;
  cudaGraph_t cap = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  e = cudaStreamGetCaptureInfo(s, &cs, nullptr, &cap, &deps, nullptr, &ndeps);
  if (e != cudaSuccess) return e;
  if (cs != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureInvalidated;
  cudaGraphConditionalHandle h;
  e = cudaGraphConditionalHandleCreate(&h, cap, 1, cudaGraphCondAssignDefault);
  if (e != cudaSuccess) return e;
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  e = cudaGraphAddNode(&node, cap, deps, nullptr, ndeps, &np);
  if (e != cudaSuccess) return e;
  e = cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
  if (e != cudaSuccess) return e;
  cudaGraph_t body = np.conditional.phGraph_out[0];
  e = cudaStreamBeginCaptureToGraph(side, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) return e;
  a.has_cond = 1;
  a.cond = h;
  cudaError_t e2 = cg_body(c, a, side);
  cudaGraph_t out_body = nullptr;
  e = cudaStreamEndCapture(side, &out_body);
  return e2 != cudaSuccess ? e2 : e;
}

}  // namespace lagh
