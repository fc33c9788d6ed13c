// Mass matrices of eq:fom.
//
// M_V (kinematic, one scalar block per component) is applied partially
// assembled.  On the Cartesian initial mesh with rho0 constant per element the
// quadrature weight rho0|J0| alpha_q is a tensor product, so the element block
// is (rho0|J0|)_K (M1 x M1 [x M1]) with M1 the 1D reference mass matrix of the
// Gauss-Lobatto basis: DIM passes of (k+1) x (k+1) contractions per component.
// Element results go to an element-local array and are gathered per node in a
// fixed order.
//
// The velocity solve is a Jacobi-preconditioned CG run by one cooperative
// persistent kernel: element phase, node gather, and vector updates separated
// by bounded grid barriers; the dot products are per-block partial sums added
// in block order by every block, so all blocks take the same decisions and the
// result is reproducible.
//
// M_E (thermodynamic, block diagonal) is applied as (rho0|J0|)_K^{-1} Mref^{-1}.
#include "device_util.cuh"

namespace lagh {

template <int DIM, int K>
struct ML {
  static constexpr int P = K + 1;
  static constexpr int ND1 = ipow(P, DIM);
  static constexpr int NT = 256;
  static constexpr int EPB = (NT / (DIM * ND1)) > 0 ? NT / (DIM * ND1) : 1;
};

// y = (M1 x M1 [x M1]) u for the DIM components of EPB elements in shared
// memory (u, y, t: [EPB][DIM][ND1]), all threads of the block.
template <int DIM, int K>
__device__ __forceinline__ void kron_mass(const double* M1, double* u, double* t, double* y,
                                          int nel) {
  using L = ML<DIM, K>;
  constexpr int P = L::P, ND1 = L::ND1;
  const int items = nel * DIM * ND1;
  // contract along x: t[.., a'] = sum_a M1[a'][a] u[.., a]
  for (int w = threadIdx.x; w < items; w += blockDim.x) {
    int ap = w % P, base = w - ap;
    double s = 0.0;
    for (int a = 0; a < P; ++a) s += M1[ap * P + a] * u[base + a];
    t[w] = s;
  }
  __syncthreads();
  if constexpr (DIM == 2) {
    for (int w = threadIdx.x; w < items; w += blockDim.x) {
      int i = w % ND1, base = w - i, a = i % P, bp = i / P;
      double s = 0.0;
      for (int b = 0; b < P; ++b) s += M1[bp * P + b] * t[base + b * P + a];
      y[w] = s;
    }
  } else {
    for (int w = threadIdx.x; w < items; w += blockDim.x) {
      int i = w % ND1, base = w - i, a = i % P, bp = (i / P) % P, cz = i / (P * P);
      double s = 0.0;
      for (int b = 0; b < P; ++b) s += M1[bp * P + b] * t[base + (cz * P + b) * P + a];
      u[w] = s;  // u is free again
    }
    __syncthreads();
    for (int w = threadIdx.x; w < items; w += blockDim.x) {
      int i = w % ND1, base = w - i, ab = i % (P * P), czp = i / (P * P);
      double s = 0.0;
      for (int cz = 0; cz < P; ++cz) s += M1[czp * P + cz] * u[base + cz * P * P + ab];
      y[w] = s;
    }
  }
  __syncthreads();
}

// Element phase of M p: ApE[el][c][i] = rho0K[el] (Kron M1) p_K for the
// elements [el0, el0 + nel).
template <int DIM, int K>
__device__ __forceinline__ void mass_elements(const Geom& g, const double* M1s,
                                              const double* __restrict__ p,
                                              const double* __restrict__ rho0K,
                                              double* __restrict__ ApE, int64_t el0, int nel,
                                              double* u, double* t, double* y) {
  using L = ML<DIM, K>;
  constexpr int P = L::P, ND1 = L::ND1;
  const int items = nel * DIM * ND1;
  for (int w = threadIdx.x; w < items; w += blockDim.x) {
    int i = w % ND1, r = w / ND1, c = r % DIM, le = r / DIM;
    int E[3] = {0, 0, 0};
    elem_ijk(g, el0 + le, E);
    int a = i % P, b = (i / P) % P, cz = DIM == 3 ? i / (P * P) : 0;
    u[w] = p[c * g.nnodes + elem_node<K>(g, E, a, b, cz)];
  }
  __syncthreads();
  kron_mass<DIM, K>(M1s, u, t, y, nel);
  for (int w = threadIdx.x; w < items; w += blockDim.x) {
    int le = w / (DIM * ND1);
    ApE[el0 * DIM * ND1 + w] = rho0K[el0 + le] * y[w];
  }
  __syncthreads();
}

template <int DIM, int K>
__global__ void __launch_bounds__(256) mass_apply_kernel(Geom g, Basis1D b,
                                                         const double* __restrict__ p,
                                                         const double* __restrict__ rho0K,
                                                         double* __restrict__ ApE) {
  using L = ML<DIM, K>;
  constexpr int P = L::P, ND1 = L::ND1, EPB = L::EPB;
  __shared__ double M1s[P * P];
  __shared__ double u[EPB * DIM * ND1], t[EPB * DIM * ND1], y[EPB * DIM * ND1];
  for (int i = threadIdx.x; i < P * P; i += blockDim.x) M1s[i] = b.M1[i / P][i % P];
  __syncthreads();
  int64_t el0 = (int64_t)blockIdx.x * EPB;
  int nel = (int)((g.nelem - el0) < EPB ? (g.nelem - el0) : EPB);
  mass_elements<DIM, K>(g, M1s, p, rho0K, ApE, el0, nel, u, t, y);
}

struct CGParams {
  Geom g;
  Basis1D b;
  const double* rhs;
  double* x;
  double *r, *z, *p, *Ap, *ApE;
  const double* dinv;
  const double* rho0K;
  double* partials;  // [3][gridDim.x]
  Barrier* bar;
  Ctl* ctl;          // iteration report and error bits
  const Ctl* gate;   // if set and done, return at once
  double rtol;
  int maxit;
};

__device__ __forceinline__ double grid_total(const double* part, int nb, double* bcast) {
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < nb; ++i) s += part[i];
    *bcast = s;
  }
  __syncthreads();
  return *bcast;
}

template <int DIM, int K>
__global__ void __launch_bounds__(256) cg_kernel(const CGParams prm) {
  using L = ML<DIM, K>;
  constexpr int P = L::P, ND1 = L::ND1, EPB = L::EPB;
  if (prm.gate != nullptr && prm.gate->done) return;
  const Geom& g = prm.g;
  __shared__ double M1s[P * P];
  __shared__ double u[EPB * DIM * ND1], t[EPB * DIM * ND1], y[EPB * DIM * ND1];
  __shared__ double red[32];
  __shared__ double bcast;
  for (int i = threadIdx.x; i < P * P; i += blockDim.x) M1s[i] = prm.b.M1[i / P][i % P];
  const int nb = gridDim.x;
  const int64_t nn = g.nnodes;
  const int64_t gstride = (int64_t)gridDim.x * blockDim.x;
  const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double* part0 = prm.partials;
  double* part1 = prm.partials + nb;
  double* part2 = prm.partials + 2 * nb;
  int* status = &prm.ctl->status;

  // r = b (free components), x = 0, z = D^{-1} r, p = z
  double l_rz = 0.0, l_bb = 0.0;
  for (int64_t node = gtid; node < nn; node += gstride) {
    int I[3];
    node_ijk(g, node, I);
    double di = prm.dinv[node];
    for (int c = 0; c < DIM; ++c) {
      int64_t k = c * nn + node;
      double bv = essential(g, I, c) ? 0.0 : prm.rhs[k];
      prm.r[k] = bv;
      prm.x[k] = 0.0;
      double zv = bv * di;
      prm.z[k] = zv;
      prm.p[k] = zv;
      l_rz += bv * zv;
      l_bb += bv * bv;
    }
  }
  {
    double s0 = block_sum(l_rz, red);
    double s1 = block_sum(l_bb, red);
    if (threadIdx.x == 0) { part0[blockIdx.x] = s0; part1[blockIdx.x] = s1; }
  }
  if (!grid_barrier(prm.bar, status)) return;
  double rz = grid_total(part0, nb, &bcast);
  const double bb = grid_total(part1, nb, &bcast);
  double rr = bb;
  int it = 0;
  bool conv = (bb == 0.0);
  const double tol2 = prm.rtol * prm.rtol * bb;
  while (!conv && it < prm.maxit) {
    ++it;
    // element phase: ApE = M_K p_K
    for (int64_t el0 = (int64_t)blockIdx.x * EPB; el0 < g.nelem; el0 += (int64_t)nb * EPB) {
      int nel = (int)((g.nelem - el0) < EPB ? (g.nelem - el0) : EPB);
      mass_elements<DIM, K>(g, M1s, prm.p, prm.rho0K, prm.ApE, el0, nel, u, t, y);
    }
    if (!grid_barrier(prm.bar, status)) return;
    // node gather, p.Ap
    double l_pap = 0.0;
    for (int64_t node = gtid; node < nn; node += gstride) {
      int I[3];
      node_ijk(g, node, I);
      for (int c = 0; c < DIM; ++c) {
        int64_t k = c * nn + node;
        double ap = essential(g, I, c) ? 0.0 : gather_node<DIM, K>(g, prm.ApE, I, c);
        prm.Ap[k] = ap;
        l_pap += prm.p[k] * ap;
      }
    }
    {
      double s = block_sum(l_pap, red);
      if (threadIdx.x == 0) part2[blockIdx.x] = s;
    }
    if (!grid_barrier(prm.bar, status)) return;
    const double pap = grid_total(part2, nb, &bcast);
    const double alpha = rz / pap;
    double l_rz2 = 0.0, l_rr = 0.0;
    for (int64_t node = gtid; node < nn; node += gstride) {
      double di = prm.dinv[node];
      for (int c = 0; c < DIM; ++c) {
        int64_t k = c * nn + node;
        prm.x[k] += alpha * prm.p[k];
        double rv = prm.r[k] - alpha * prm.Ap[k];
        prm.r[k] = rv;
        double zv = rv * di;
        prm.z[k] = zv;
        l_rz2 += rv * zv;
        l_rr += rv * rv;
      }
    }
    {
      double s0 = block_sum(l_rz2, red);
      double s1 = block_sum(l_rr, red);
      if (threadIdx.x == 0) { part0[blockIdx.x] = s0; part1[blockIdx.x] = s1; }
    }
    if (!grid_barrier(prm.bar, status)) return;
    const double rz_new = grid_total(part0, nb, &bcast);
    rr = grid_total(part1, nb, &bcast);
    if (rr <= tol2) { conv = true; break; }
    if (!(rr == rr)) break;  // NaN: give up, reported as not converged
    const double beta = rz_new / rz;
    rz = rz_new;
    for (int64_t node = gtid; node < nn; node += gstride)
      for (int c = 0; c < DIM; ++c) {
        int64_t k = c * nn + node;
        prm.p[k] = prm.z[k] + beta * prm.p[k];
      }
    if (!grid_barrier(prm.bar, status)) return;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    prm.ctl->cg_last_iters = it;
    prm.ctl->cg_last_relres = bb > 0.0 ? sqrt(rr / bb) : 0.0;
    prm.ctl->cg_iters += it;
    if (!conv) atomicOr(status, kDevCG);
  }
}

template <int DIM, int K>
__global__ void mass_solve_e_kernel(Geom g, Basis1D b, const double* __restrict__ rhs,
                                    const double* __restrict__ rho0K, double* __restrict__ out) {
  constexpr int ND2 = ipow(K, DIM);
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= g.ne) return;
  int64_t el = idx / ND2;
  int j = (int)(idx - el * ND2);
  double s = 0.0;
  for (int l = 0; l < ND2; ++l) s += b.MEinv[j * ND2 + l] * rhs[el * ND2 + l];
  out[idx] = s / rho0K[el];
}

// Partial sums of v.(M_V v) (from the gathered Mv) and 1.M_E e per block.
template <int DIM, int K>
__global__ void energy_partials_kernel(Geom g, Basis1D b, const double* __restrict__ v,
                                       const double* __restrict__ Mv, const double* __restrict__ e,
                                       const double* __restrict__ rho0K, double* __restrict__ part) {
  constexpr int ND2 = ipow(K, DIM);
  __shared__ double red[32];
  double ke = 0.0, ie = 0.0;
  int64_t gstride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < g.nv; i += gstride)
    ke += v[i] * Mv[i];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < g.ne; i += gstride) {
    int64_t el = i / ND2;
    ie += rho0K[el] * b.L2int[i - el * ND2] * e[i];
  }
  double s0 = block_sum(ke, red);
  double s1 = block_sum(ie, red);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = s0;
    part[2 * blockIdx.x + 1] = s1;
  }
}

__global__ void energy_final_kernel(const double* part, int nb, double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double ke = 0.0, ie = 0.0;
    for (int i = 0; i < nb; ++i) {
      ke += part[2 * i];
      ie += part[2 * i + 1];
    }
    *out = 0.5 * ke + ie;
  }
}

// ---------------------------------------------------------- launchers ----

#define LAGH_DISPATCH_M(DIMV, KV, FN, ...)                  \
  do {                                                      \
    if ((DIMV) == 2 && (KV) == 1) return FN<2, 1>(__VA_ARGS__); \
    if ((DIMV) == 2 && (KV) == 2) return FN<2, 2>(__VA_ARGS__); \
    if ((DIMV) == 2 && (KV) == 3) return FN<2, 3>(__VA_ARGS__); \
    if ((DIMV) == 3 && (KV) == 1) return FN<3, 1>(__VA_ARGS__); \
    if ((DIMV) == 3 && (KV) == 2) return FN<3, 2>(__VA_ARGS__); \
    return cudaErrorInvalidValue;                           \
  } while (0)

template <int DIM, int K>
static cudaError_t mass_apply_dk(const lh_ctx* c, const double* in, double* out, cudaStream_t s) {
  using L = ML<DIM, K>;
  int64_t blocks = (c->g.nelem + L::EPB - 1) / L::EPB;
  mass_apply_kernel<DIM, K><<<(unsigned)blocks, L::NT, 0, s>>>(c->g, c->basis, in, c->a.rho0K,
                                                                 c->a.ApE);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_gather(c, c->a.ApE, out, 1.0, 0, nullptr, s);
}

cudaError_t launch_mass_apply(const lh_ctx* c, const double* in, double* out, cudaStream_t s) {
  LAGH_DISPATCH_M(c->g.dim, c->g.k, mass_apply_dk, c, in, out, s);
}

template <int DIM, int K>
static cudaError_t cg_occ_dk(lh_ctx* c) {
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cg_kernel<DIM, K>, 256, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  using L = ML<DIM, K>;
  int64_t want_el = (c->g.nelem + L::EPB - 1) / L::EPB;
  int64_t want_nd = (c->g.nnodes + 255) / 256;
  int64_t want = want_el > want_nd ? want_el : want_nd;
  int64_t cap = (int64_t)per_sm * c->num_sms;
  c->cg_blocks = (int)(want < cap ? want : cap);
  if (c->cg_blocks < 1) c->cg_blocks = 1;
  c->cg_threads = 256;
  return cudaSuccess;
}

cudaError_t cg_occupancy(lh_ctx* c) { LAGH_DISPATCH_M(c->g.dim, c->g.k, cg_occ_dk, c); }

template <int DIM, int K>
static cudaError_t cg_dk(const lh_ctx* c, const double* rhs, double* out, const Ctl* gate,
                         cudaStream_t s) {
  CGParams prm;
  prm.g = c->g;
  prm.b = c->basis;
  prm.rhs = rhs;
  prm.x = out;
  prm.r = c->a.r;
  prm.z = c->a.z;
  prm.p = c->a.p;
  prm.Ap = c->a.Ap;
  prm.ApE = c->a.ApE;
  prm.dinv = c->a.dinv;
  prm.rho0K = c->a.rho0K;
  prm.partials = c->a.partials;
  prm.bar = c->a.bar;
  prm.ctl = c->a.ctl;
  prm.gate = gate;
  prm.rtol = c->cg_rtol;
  prm.maxit = c->cg_maxit;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)c->cg_blocks);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, cg_kernel<DIM, K>, prm);
}

cudaError_t launch_cg(const lh_ctx* c, const double* rhs, double* out, const Ctl* gate,
                      cudaStream_t s) {
  LAGH_DISPATCH_M(c->g.dim, c->g.k, cg_dk, c, rhs, out, gate, s);
}

template <int DIM, int K>
static cudaError_t mse_dk(const lh_ctx* c, const double* rhs, double* out, cudaStream_t s) {
  int64_t blocks = (c->g.ne + 255) / 256;
  mass_solve_e_kernel<DIM, K><<<(unsigned)blocks, 256, 0, s>>>(c->g, c->basis, rhs, c->a.rho0K, out);
  return cudaGetLastError();
}

cudaError_t launch_mass_solve_e(const lh_ctx* c, const double* rhs, double* out, cudaStream_t s) {
  LAGH_DISPATCH_M(c->g.dim, c->g.k, mse_dk, c, rhs, out, s);
}

template <int DIM, int K>
static cudaError_t energy_dk(const lh_ctx* c, const double* v, const double* e, double* out,
                             cudaStream_t s) {
  cudaError_t err = launch_mass_apply(c, v, c->a.tmpV, s);
  if (err != cudaSuccess) return err;
  const int nb = 256;
  energy_partials_kernel<DIM, K><<<nb, 256, 0, s>>>(c->g, c->basis, v, c->a.tmpV, e, c->a.rho0K,
                                                    c->a.partials);
  energy_final_kernel<<<1, 32, 0, s>>>(c->a.partials, nb, out);
  return cudaGetLastError();
}

cudaError_t launch_total_energy(const lh_ctx* c, const double* v, const double* e, double* out,
                                cudaStream_t s) {
  LAGH_DISPATCH_M(c->g.dim, c->g.k, energy_dk, c, v, e, out, s);
}

}  // namespace lagh
