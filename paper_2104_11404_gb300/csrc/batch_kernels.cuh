// Device side of the batched form: many independent instances of the time
// step (the parameter sweep whose states are the snapshots of Section 4),
// each on its own Cartesian box mesh, advanced together.
//
// One persistent kernel per RK stage.  Every CTA takes instances from a queue
// ordered largest first and runs the whole stage of an instance alone: force
// tiles, node gather, velocity solve, velocity / position update, energy
// update and, after the second stage, the step control and commit.  Inside an
// instance the only synchronisation is __syncthreads, so an instance never
// waits on another CTA.
//
// Velocity solve.  rho0 |J0| is the same in every element of an instance, so
// the kinematic mass matrix restricted to the free entries of component c is
// rho0|J0| times the Kronecker product of assembled 1D reference mass matrices
// (along direction c without its two end nodes, the wall-normal condition).
// Its exact inverse -- banded Cholesky solves along every node line, FP64 --
// preconditions the CG on the partially assembled operator, so the solve
// stops after its first residual check.
#pragma once

#include "control.cuh"
#include "force_tiles.cuh"
#include "line_solve.cuh"
#include "mass_ops.cuh"

namespace lagh {

struct BInst {
  Geom g;
  Phys ph;
  CtlConsts kc;
  double rho0K;         // rho0 |J0| of every element of the instance
  double scale;         // 1 / rho0K
  int64_t ov, oe, oel;  // offsets in the packed N_V-, N_E- and per-element arrays
  int64_t fac[3][2];    // offsets (doubles) of the 1D Cholesky tables [direction][variant]
  int64_t pad;
};

// Every pointer is device memory.  Scratch arrays are per CTA (slot =
// blockIdx.x), each slot `s_*` entries long.
struct BatchArgs {
  const BInst* inst;
  const int32_t* order;  // instance ids, largest first
  int32_t n;
  Ctl* ctl;              // one control block per instance
  double *v, *e, *x, *vh, *eh, *xh, *vn, *en, *xn, *vbar;
  const double* rho0K;   // per element (packed by oel)
  const double* rho0Kinv;
  const double* fac;     // line-solve tables (see line_solve)
  double* F1E;           // element rows of F.1, then of M p (CG)
  float* FK;             // mixed: element force matrices
  double* D;             // FP64: stress weights
  double* srcE;          // energy source (2D Taylor-Green)
  double* vec;           // CG vectors: r (= rhs), x, z, p, Ap
  int64_t s_f1e, s_fkd, s_src, s_vec;
  unsigned int* qctr;    // queue counters [0..3] and exit tickets [4..7]
  int* ndone;            // instances that finished during the current run
  double rtol;
  int maxit;
  int smem_lines;        // line solves staged in shared memory
  // sampled force / energy / estimate arguments
  const int64_t* list_off;
  const int32_t* list;
  const double* vtest;
  double* out;           // element rows (sampled force), energies or estimates
  double* out2;          // sampled F^T w rows
  // snapshot capture (Section 4): caller-owned column-major matrices; per
  // instance the offset (doubles) of its first column in Sv / Sx and in Se
  // (-1: not captured) and the count of snapshots taken
  double *Sv, *Se, *Sx;
  const int64_t* snap_ov;
  const int64_t* snap_oe;
  int64_t* snap_count;
  int64_t snap_cap;
};

enum { kQStage0 = 0, kQStage1 = 1, kQAux = 2 };

// Next instance of queue q for this CTA (all threads), or -1 when it is empty.
// The last CTA to find the queue empty resets it for the next launch.
__device__ __forceinline__ int next_instance(const BatchArgs& a, int q) {
  __shared__ int s_q;
  __syncthreads();
  if (threadIdx.x == 0) {
    int k = (int)atomicAdd(&a.qctr[q], 1u);
    if (k >= a.n) {
      k = -1;
      if (atomicAdd(&a.qctr[4 + q], 1u) == gridDim.x - 1) {
        a.qctr[q] = 0u;
        a.qctr[4 + q] = 0u;
      }
    } else {
      k = a.order[k];
    }
    s_q = k;
  }
  __syncthreads();
  return s_q;
}

// Sum over the CTA in a fixed order, returned to every thread.
__device__ __forceinline__ double cta_sum(double v) {
  __shared__ double sh[32];
  __shared__ double res;
  double s = block_sum(v, sh);
  if (threadIdx.x == 0) res = s;
  __syncthreads();
  return res;
}

// The instance descriptor, copied to shared memory by the CTA.
__device__ __forceinline__ void load_instance(const BatchArgs& a, int i, BInst* sI) {
  const int words = (int)(sizeof(BInst) / sizeof(int64_t));
  const int64_t* src = reinterpret_cast<const int64_t*>(a.inst + i);
  int64_t* dst = reinterpret_cast<int64_t*>(sI);
  for (int w = threadIdx.x; w < words; w += blockDim.x) dst[w] = src[w];
  __syncthreads();
}

// Multi-index of a node of an instance (32-bit: an instance of the batched
// form holds fewer than 2^31 velocity unknowns).
__device__ __forceinline__ void node_ijk32(const Geom& g, int node, int I[3]) {
  const int n0 = g.nn[0], n1 = g.nn[1];
  const int r = node / n0;
  I[0] = node - r * n0;
  I[1] = r % n1;
  I[2] = r / n1;
}

// z_c = scale (G^-1 (x) ... (x) G^-1) r_c on the free entries of component c
// (zero on its wall-normal nodes) for every component: the 1D solves along
// each direction in turn, every node line independent.  mode 2: all
// components staged in buf (DIM nnodes doubles of shared memory) and solved
// together; mode 1: one component at a time in buf (nnodes doubles); mode 0:
// in place on z in device memory.  With Pv and rz given, the copy-out also
// sets Pv = z and adds this thread's share of r . z to *rz.
template <int DIM, int K>
__device__ void tensor_solve(const Geom& g, const double* __restrict__ fac,
                             const int64_t (*fo)[2], double scale, const double* r, double* z,
                             double* buf, int mode, double* Pv = nullptr, double* rz = nullptr) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int nn = (int)g.nnodes;
  const int cpass = mode == 2 ? DIM : 1;  // components per pass
  double rzl = 0.0;
  for (int c0 = 0; c0 < DIM; c0 += cpass) {
    double* w = mode == 0 ? z + (int64_t)c0 * nn : buf;  // holds components c0 .. c0 + cpass - 1
    for (int node = tid; node < nn; node += nt) {
      int I[3];
      node_ijk32(g, node, I);
      for (int cc = 0; cc < cpass; ++cc) {
        const int c = c0 + cc;
        w[cc * nn + node] = (I[c] == 0 || I[c] == g.nn[c] - 1) ? 0.0 : r[c * nn + node];
      }
    }
    __syncthreads();
    for (int d = 0; d < DIM; ++d) {
      const int nlines = nn / g.nn[d];
      const int64_t stride = d == 0 ? 1 : (d == 1 ? (int64_t)g.nn[0] : (int64_t)g.nn[0] * g.nn[1]);
      for (int li = tid; li < cpass * nlines; li += nt) {
        const int cc = li / nlines, c = c0 + cc;
        const int line = li - cc * nlines;
        const int var = (d == c) ? 1 : 0;
        int I[3] = {0, 0, 0};
        if (d == 0) { I[1] = line % g.nn[1]; I[2] = line / g.nn[1]; }
        else if (d == 1) { I[0] = line % g.nn[0]; I[2] = line / g.nn[0]; }
        else { I[0] = line % g.nn[0]; I[1] = line / g.nn[0]; }
        if (d != c && (I[c] == 0 || I[c] == g.nn[c] - 1)) continue;  // essential line
        line_solve<K>(w + (int64_t)cc * nn + node_index(g, I[0], I[1], I[2]) + var * stride,
                      stride, g.nn[d] - 2 * var, fac + fo[d][var]);
      }
      __syncthreads();
    }
    const int64_t o = (int64_t)c0 * nn;
    if (Pv != nullptr) {
      for (int idx = tid; idx < cpass * nn; idx += nt) {
        const double zv = scale * w[idx];
        z[o + idx] = zv;
        Pv[o + idx] = zv;
        rzl = fma(r[o + idx], zv, rzl);
      }
    } else {
      for (int idx = tid; idx < cpass * nn; idx += nt) z[o + idx] = scale * w[idx];
    }
    __syncthreads();
  }
  if (rz != nullptr) *rz = rzl;
}

// Shared-memory plan of the stage kernel (bytes of each phase; the phases
// reuse one dynamic buffer).  QPT: quadrature points per thread of the force
// tiles.
template <int DIM, int K, bool MIXED, int NTT, int QPT = 1>
struct BL {
  using F = FL<DIM, K, MIXED, NTT, QPT>;
  using E = EL<DIM, K, MIXED, NTT>;
  static constexpr int P = K + 1, ND1 = ipow(P, DIM), ND2 = ipow(K, DIM), NQD = ipow(2 * K, DIM);
  static constexpr int CGT = (NTT / (DIM * ND1)) > 0 ? NTT / (DIM * ND1) : 1;  // elements per mass tile
  static constexpr size_t B_MASS = (size_t)(3 * CGT * DIM * ND1 + P * P) * sizeof(double);
  static constexpr size_t B_FIXED = F::BYTES > E::BYTES ? (F::BYTES > B_MASS ? F::BYTES : B_MASS)
                                                        : (E::BYTES > B_MASS ? E::BYTES : B_MASS);
  // bytes with the line buffer after the mass tile: DIM (smem_lines = 2), one
  // (1) or no (0) components of nnodes doubles
  static size_t bytes(int64_t nnodes_max, int smem_lines) {
    const int comps = smem_lines == 2 ? DIM : (smem_lines == 1 ? 1 : 0);
    size_t cg = B_MASS + (size_t)comps * nnodes_max * sizeof(double);
    return cg > B_FIXED ? cg : B_FIXED;
  }
};

// A p for the CG of a 2D instance, with p and the node sums in shared memory
// (buf: 2 nnodes doubles), one component at a time: every element's
// (M1 x M1) p_K is formed in registers and added to its nodes.  The elements
// are taken in four colours (parity of the element indices), so no two
// elements of one colour share a node and every node receives its (at most
// four) contributions in colour order: the sums are deterministic.  The
// second factor's table M1r is rho0 |J0| M1 (uniform in an instance) and its
// products are accumulated onto the node sums directly.  Writes AP (zero on
// the wall-normal entries) and returns p . Ap.
template <int K>
__device__ double cta_mass_colored(const Geom& g, const double* M1s, const double* M1r,
                                   const double* Pv, double* AP, double* buf) {
  constexpr int P = K + 1;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int nn = (int)g.nnodes, n0 = g.nn[0];
  double* pc = buf;
  double* ac = buf + nn;
  double pap = 0.0;
  for (int c = 0; c < 2; ++c) {
    for (int node = tid; node < nn; node += nt) {
      pc[node] = Pv[c * nn + node];
      ac[node] = 0.0;
    }
    __syncthreads();
    for (int color = 0; color < 4; ++color) {
      const int bx = color & 1, by = color >> 1;
      const int mx = (g.n[0] - bx + 1) / 2, my = (g.n[1] - by + 1) / 2;
      for (int item = tid; item < mx * my; item += nt) {
        const int iy = item / mx;
        const int ex = 2 * (item - iy * mx) + bx, ey = 2 * iy + by;
        const int base = ex * K + n0 * (ey * K);
        double t[P][P];
#pragma unroll
        for (int b = 0; b < P; ++b) {
          double u[P];
#pragma unroll
          for (int a = 0; a < P; ++a) u[a] = pc[base + n0 * b + a];
#pragma unroll
          for (int ap = 0; ap < P; ++ap) {
            double acc = 0.0;
#pragma unroll
            for (int a = 0; a < P; ++a) acc = fma(M1s[ap * P + a], u[a], acc);
            t[b][ap] = acc;
          }
        }
#pragma unroll
        for (int bp = 0; bp < P; ++bp)
#pragma unroll
          for (int ap = 0; ap < P; ++ap) {
            double acc = ac[base + n0 * bp + ap];
#pragma unroll
            for (int b = 0; b < P; ++b) acc = fma(M1r[bp * P + b], t[b][ap], acc);
            ac[base + n0 * bp + ap] = acc;
          }
      }
      __syncthreads();
    }
    for (int node = tid; node < nn; node += nt) {
      const int i1 = node / n0, i0 = node - i1 * n0;
      const int ic = c == 0 ? i0 : i1;
      const double ap = (ic == 0 || ic == g.nn[c] - 1) ? 0.0 : ac[node];
      AP[c * nn + node] = ap;
      pap = fma(pc[node], ap, pap);
    }
    __syncthreads();
  }
  return cta_sum(pap);
}

// In-CTA preconditioned CG: M_V x = b on the free components, b in R (the
// essential entries of b are zero), x in X.  Returns the iteration count;
// *relres = ||r|| / ||b||; *conv = converged.  R, X, Z, Pv, AP and ApE are
// disjoint (slices of the CTA's scratch slot, and its element buffer), which
// lets the vector loops issue later iterations' loads ahead of their stores.
template <int DIM, int K, int NTT>
__device__ int cta_cg(const BatchArgs& a, const BInst& I, double* __restrict__ R,
                      double* __restrict__ X, double* __restrict__ Z, double* __restrict__ Pv,
                      double* __restrict__ AP, double* __restrict__ ApE,
                      const double* __restrict__ rho0K, unsigned char* smem, const double* M1,
                      double* relres, bool* conv) {
  using L = BL<DIM, K, false, NTT>;
  constexpr int P = K + 1, ND1 = ipow(P, DIM), CGT = L::CGT;
  const Geom& g = I.g;
  const int tid = threadIdx.x;
  const int64_t nv = g.nv, nn = g.nnodes;
  double* M1s = reinterpret_cast<double*>(smem);
  double* u = M1s + P * P;
  double* t = u + CGT * DIM * ND1;
  double* y = t + CGT * DIM * ND1;
  double* lines = a.smem_lines ? y + CGT * DIM * ND1 : nullptr;
  double* M1r = t;  // 2D shared-memory apply: rho0 |J0| M1 (the tile buffers are unused there)
  for (int i = tid; i < P * P; i += NTT) {
    const double m = M1[(i / P) * (kMaxOrder + 1) + i % P];
    M1s[i] = m;
    M1r[i] = I.rho0K * m;
  }
  double bb = 0.0;
#pragma unroll 4
  for (int64_t k = tid; k < nv; k += NTT) {
    const double bv = R[k];
    X[k] = 0.0;
    bb += bv * bv;
  }
  bb = cta_sum(bb);
  if (!(bb > 0.0)) {
    *relres = 0.0;
    *conv = true;
    return 0;
  }
  double rz;
  tensor_solve<DIM, K>(g, a.fac, I.fac, I.scale, R, Z, lines, a.smem_lines, Pv, &rz);
  rz = cta_sum(rz);
  int it = 0;
  double rr = bb;
  bool ok = false;
  while (true) {
    ++it;
    double pap;
    if (DIM == 2 && a.smem_lines == 2) {
      // A p on shared-memory node arrays (rho0 |J0| is uniform in an instance)
      pap = cta_mass_colored<K>(g, M1s, M1r, Pv, AP, lines);
    } else {
      // element phase (tiles of CGT elements), then the node gather
      for (int64_t el0 = 0; el0 < g.nelem; el0 += CGT) {
        const int nel = (int)((g.nelem - el0) < CGT ? (g.nelem - el0) : CGT);
        mass_elements<DIM, K>(g, M1s, Pv, rho0K, ApE, el0, nel, u, t, y);
      }
      pap = 0.0;
      for (int node = tid; node < (int)nn; node += NTT) {
        int Ix[3];
        node_ijk32(g, node, Ix);
        for (int c = 0; c < DIM; ++c) {
          const int64_t k = c * nn + node;
          const double ap = essential(g, Ix, c) ? 0.0 : gather_node<DIM, K>(g, ApE, Ix, c);
          AP[k] = ap;
          pap += Pv[k] * ap;
        }
      }
      pap = cta_sum(pap);
    }
    const double alpha = rz / pap;
    double lrr = 0.0;
#pragma unroll 4
  for (int64_t k = tid; k < nv; k += NTT) {
      X[k] += alpha * Pv[k];
      const double rv = R[k] - alpha * AP[k];
      R[k] = rv;
      lrr += rv * rv;
    }
    rr = cta_sum(lrr);
    ok = rr <= a.rtol * a.rtol * bb;
    if (ok || !(rr == rr) || it >= a.maxit) break;
    tensor_solve<DIM, K>(g, a.fac, I.fac, I.scale, R, Z, lines, a.smem_lines);
    double lrz = 0.0;
#pragma unroll 4
  for (int64_t k = tid; k < nv; k += NTT) lrz += R[k] * Z[k];
    const double rz_new = cta_sum(lrz);
    const double beta = rz_new / rz;
    rz = rz_new;
#pragma unroll 4
  for (int64_t k = tid; k < nv; k += NTT) Pv[k] = Z[k] + beta * Pv[k];
    __syncthreads();
  }
  *relres = sqrt(rr / bb);
  *conv = ok;
  return it;
}

// One RK2-average stage of every unfinished instance (stage 0: S^n ->
// S^{n+1/2}; stage 1: S^{n+1/2} -> candidate S^{n+1}, control, commit).
template <int DIM, int K, bool MIXED, int NTT, int QPT>
__global__ void __launch_bounds__(NTT) batch_stage_kernel(const BatchArgs a, const Basis1D bas,
                                                          int stage) {
  using F = FL<DIM, K, MIXED, NTT, QPT>;
  using E = EL<DIM, K, MIXED, NTT>;
  constexpr int ND1 = F::ND1;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ BInst sI;
  __shared__ unsigned long long s_tau;
  __shared__ int s_status, s_skip, s_acc;
  __shared__ long long s_snap;
  __shared__ double s_dt;
  const int tid = threadIdx.x;
  const int64_t slot = blockIdx.x;
  double* F1E = a.F1E + slot * a.s_f1e;
  float* FK = MIXED ? a.FK + slot * a.s_fkd : nullptr;
  double* D = MIXED ? nullptr : a.D + slot * a.s_fkd;
  double* srcE = a.srcE ? a.srcE + slot * a.s_src : nullptr;
  double* vec = a.vec + slot * a.s_vec;
  const int q = stage == 0 ? kQStage0 : kQStage1;
  for (int i = next_instance(a, q); i >= 0; i = next_instance(a, q)) {
    Ctl* ctl = a.ctl + i;
    if (tid == 0) {
      s_skip = ctl->done;
      s_dt = ctl->dt_use;
      s_tau = kInfBits;
      s_status = 0;
    }
    load_instance(a, i, &sI);  // synchronises
    if (s_skip) continue;
    const Geom& g = sI.g;
    const double* rho0K = a.rho0K + sI.oel;
    const double* vs = (stage == 0 ? a.v : a.vh) + sI.ov;
    const double* xs = (stage == 0 ? a.x : a.xh) + sI.ov;
    const double* es = (stage == 0 ? a.e : a.eh) + sI.oe;
    // ---- force: F.1 rows, element matrices / stress weights, estimate ----
    ForceArgs fa = {};
    fa.v = vs; fa.e = es; fa.x = xs;
    fa.nslots = g.nelem;
    fa.F1E = F1E;
    fa.D = D;
    fa.FK = FK;
    fa.srcE = (sI.ph.source && srcE) ? srcE : nullptr;
    fa.tau_bits = &s_tau;
    fa.status = &s_status;
    fa.mode = kForceFull;
    force_tables<DIM, K, MIXED, NTT, QPT>(bas, smem);
    __syncthreads();
    for (int64_t el0 = 0; el0 < g.nelem; el0 += F::EPB)
      force_tile<DIM, K, MIXED, NTT, QPT>(g, sI.ph, bas, fa, rho0K, smem, el0);
    __syncthreads();
    if (tid == 0) {
      ctl->tau_bits[stage] = s_tau;
      ctl->status |= s_status;
    }
    // ---- momentum right-hand side -F.1 (wall components zero) ----
    double* R = vec;
    double* X = vec + g.nv;
    double* Z = vec + 2 * g.nv;
    double* Pv = vec + 3 * g.nv;
    double* AP = vec + 4 * g.nv;
    for (int node = tid; node < (int)g.nnodes; node += NTT) {
      int Ix[3];
      node_ijk32(g, node, Ix);
      for (int c = 0; c < DIM; ++c)
        R[c * g.nnodes + node] = essential(g, Ix, c) ? 0.0 : -gather_node<DIM, K>(g, F1E, Ix, c);
    }
    __syncthreads();
    // ---- acceleration: M_V a = -F.1 ----
    double relres;
    bool conv;
    const int its = cta_cg<DIM, K, NTT>(a, sI, R, X, Z, Pv, AP, F1E, rho0K, smem, &bas.M1[0][0],
                                        &relres, &conv);
    if (tid == 0) {
      ctl->cg_iters += its;
      ctl->cg_last_iters = its;
      ctl->cg_last_relres = relres;
      if (!conv) ctl->status |= kDevCG;
    }
    // ---- velocity and position ----
    const double dt = s_dt;
    const double* v0 = a.v + sI.ov;
    const double* x0 = a.x + sI.ov;
    if (stage == 0) {
      double* vh = a.vh + sI.ov;
      double* xh = a.xh + sI.ov;
      for (int64_t k = tid; k < g.nv; k += NTT) {
        const double vhalf = v0[k] + 0.5 * dt * X[k];
        vh[k] = vhalf;
        xh[k] = x0[k] + 0.5 * dt * vhalf;
      }
    } else {
      double* vn = a.vn + sI.ov;
      double* vb = a.vbar + sI.ov;
      double* xn = a.xn + sI.ov;
      for (int64_t k = tid; k < g.nv; k += NTT) {
        const double v1 = v0[k] + dt * X[k];
        const double vbar = 0.5 * (v0[k] + v1);
        vn[k] = v1;
        vb[k] = vbar;
        xn[k] = x0[k] + dt * vbar;
      }
    }
    __syncthreads();
    // ---- energy: e_out = e^n + c dt M_E^-1 (F^T w + src) ----
    EnergyArgs ea = {};
    ea.w = (stage == 0 ? a.vh : a.vbar) + sI.ov;
    ea.D = D;
    ea.FK = FK;
    ea.srcE = fa.srcE;
    ea.e_base = a.e + sI.oe;
    ea.e_out = (stage == 0 ? a.eh : a.en) + sI.oe;
    ea.frac = stage == 0 ? 0.5 : 1.0;
    ea.dt = dt;
    ea.ctl = nullptr;
    ea.rho0Kinv = a.rho0Kinv + sI.oel;
    energy_tables<DIM, K, MIXED, NTT>(bas, smem);
    __syncthreads();
    for (int64_t el0 = 0; el0 < g.nelem; el0 += E::EPB)
      energy_tile<DIM, K, MIXED, NTT>(g, bas, ea, rho0K, smem, el0);
    __syncthreads();
    if (stage == 0) continue;
    // ---- step control and commit ----
    if (tid == 0) {
      control_update(ctl, sI.kc);
      s_acc = ctl->accepted;
      if (ctl->done) atomicAdd(a.ndone, 1);
    }
    __syncthreads();
    if (s_acc) {
      double* v = a.v + sI.ov;
      double* x = a.x + sI.ov;
      double* e = a.e + sI.oe;
      const double* vn = a.vn + sI.ov;
      const double* xn = a.xn + sI.ov;
      const double* en = a.en + sI.oe;
      for (int64_t k = tid; k < g.nv; k += NTT) {
        v[k] = vn[k];
        x[k] = xn[k];
      }
      for (int64_t k = tid; k < g.ne; k += NTT) e[k] = en[k];
      // snapshots of the accepted step: S^{n+1/2}, then S^{n+1}
      if (a.snap_count != nullptr && a.snap_ov[i] >= 0) {
        if (tid == 0) {
          s_snap = a.snap_count[i];
          a.snap_count[i] = s_snap + 2;
        }
        __syncthreads();
        const int64_t c0 = s_snap;
        const double* vh = a.vh + sI.ov;
        const double* xh = a.xh + sI.ov;
        const double* eh = a.eh + sI.oe;
        for (int h = 0; h < 2; ++h) {
          if (c0 + h >= a.snap_cap) break;
          double* sv = a.Sv + a.snap_ov[i] + (c0 + h) * g.nv;
          double* sx = a.Sx + a.snap_ov[i] + (c0 + h) * g.nv;
          double* se = a.Se + a.snap_oe[i] + (c0 + h) * g.ne;
          for (int64_t k = tid; k < g.nv; k += NTT) {
            sv[k] = h == 0 ? vh[k] : vn[k];
            sx[k] = h == 0 ? xh[k] : xn[k];
          }
          for (int64_t k = tid; k < g.ne; k += NTT) se[k] = h == 0 ? eh[k] : en[k];
        }
      }
    }
    (void)ND1;
  }
}

// Estimate of every instance's current state (ordered bits into out[i]) and
// its error flags (ctl status), for the first step size of a run.
template <int DIM, int K, bool MIXED, int NTT>
__global__ void __launch_bounds__(NTT) batch_estimate_kernel(const BatchArgs a, const Basis1D bas) {
  using F = FL<DIM, K, MIXED, NTT>;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ BInst sI;
  __shared__ unsigned long long s_tau;
  __shared__ int s_status;
  double* F1E = a.F1E + (int64_t)blockIdx.x * a.s_f1e;
  force_tables<DIM, K, MIXED, NTT>(bas, smem);  // next_instance synchronises
  for (int i = next_instance(a, kQAux); i >= 0; i = next_instance(a, kQAux)) {
    if (threadIdx.x == 0) {
      s_tau = kInfBits;
      s_status = 0;
    }
    load_instance(a, i, &sI);
    const Geom& g = sI.g;
    ForceArgs fa = {};
    fa.v = a.v + sI.ov; fa.e = a.e + sI.oe; fa.x = a.x + sI.ov;
    fa.nslots = g.nelem;
    fa.F1E = F1E;
    fa.tau_bits = &s_tau;
    fa.status = &s_status;
    fa.mode = kForceFull;
    for (int64_t el0 = 0; el0 < g.nelem; el0 += F::EPB)
      force_tile<DIM, K, MIXED, NTT>(g, sI.ph, bas, fa, a.rho0K + sI.oel, smem, el0);
    __syncthreads();
    if (threadIdx.x == 0) {
      reinterpret_cast<unsigned long long*>(a.out)[i] = s_tau;
      a.ctl[i].status |= (s_status & kDevNonFinite);
    }
  }
}

// Restricted force of each instance on its listed elements (Section 3.3):
// element rows of F.1 into out (and of F^T w into out2) in list order, packed
// by list_off, and the estimate over the listed elements (ordered bits, 0 for
// an inverted element) into est[i].
template <int DIM, int K, bool MIXED, int NTT>
__global__ void __launch_bounds__(NTT) batch_sampled_kernel(const BatchArgs a, const Basis1D bas,
                                                            unsigned long long* est) {
  using F = FL<DIM, K, MIXED, NTT>;
  constexpr int ND1 = F::ND1, ND2 = F::ND2;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ BInst sI;
  __shared__ unsigned long long s_tau;
  __shared__ int s_status;
  force_tables<DIM, K, MIXED, NTT>(bas, smem);  // next_instance synchronises
  for (int i = next_instance(a, kQAux); i >= 0; i = next_instance(a, kQAux)) {
    if (threadIdx.x == 0) {
      s_tau = kInfBits;
      s_status = 0;
    }
    load_instance(a, i, &sI);
    const Geom& g = sI.g;
    const int64_t o = a.list_off[i], cnt = a.list_off[i + 1] - o;
    ForceArgs fa = {};
    fa.v = a.v + sI.ov; fa.e = a.e + sI.oe; fa.x = a.x + sI.ov;
    fa.vtest = a.vtest ? a.vtest + sI.ov : nullptr;
    fa.list = a.list + o;
    fa.nslots = cnt;
    fa.F1E = a.out + o * DIM * ND1;
    fa.FTvE = a.out2 ? a.out2 + o * ND2 : nullptr;
    fa.tau_bits = &s_tau;
    fa.status = &s_status;
    fa.mode = kForceFull;
    for (int64_t s0 = 0; s0 < cnt; s0 += F::EPB)
      force_tile<DIM, K, MIXED, NTT>(g, sI.ph, bas, fa, a.rho0K + sI.oel, smem, s0);
    __syncthreads();
    if (threadIdx.x == 0) est[i] = (s_status & kDevTangled) ? 0ull : s_tau;
  }
}

// Total energy 1/2 v.M_V.v + 1.M_E.e of every instance (element sums in a
// fixed order) into out[i].
template <int DIM, int K, int NTT>
__global__ void __launch_bounds__(NTT) batch_energy_kernel(const BatchArgs a, const Basis1D bas) {
  constexpr int P = K + 1, ND1 = ipow(P, DIM), ND2 = ipow(K, DIM);
  constexpr int CGT = BL<DIM, K, false, NTT>::CGT;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ BInst sI;
  double* M1s = reinterpret_cast<double*>(smem);
  double* u = M1s + P * P;
  double* t = u + CGT * DIM * ND1;
  double* y = t + CGT * DIM * ND1;
  double* vc = y + CGT * DIM * ND1;
  for (int i = threadIdx.x; i < P * P; i += NTT) M1s[i] = bas.M1[i / P][i % P];
  for (int i = next_instance(a, kQAux); i >= 0; i = next_instance(a, kQAux)) {
    load_instance(a, i, &sI);
    const Geom& g = sI.g;
    const double* v = a.v + sI.ov;
    const double* e = a.e + sI.oe;
    const double* rho0K = a.rho0K + sI.oel;
    double ke = 0.0, ie = 0.0;
    for (int64_t el0 = 0; el0 < g.nelem; el0 += CGT) {
      const int nel = (int)((g.nelem - el0) < CGT ? (g.nelem - el0) : CGT);
      const int items = nel * DIM * ND1;
      for (int w = threadIdx.x; w < items; w += NTT) {
        int ii = w % ND1, r = w / ND1, c = r % DIM, le = r / DIM;
        int Ee[3] = {0, 0, 0};
        elem_ijk(g, el0 + le, Ee);
        int aa = ii % P, b = (ii / P) % P, cz = DIM == 3 ? ii / (P * P) : 0;
        const double val = v[c * g.nnodes + elem_node<K>(g, Ee, aa, b, cz)];
        u[w] = val;
        vc[w] = val;
      }
      __syncthreads();
      kron_mass<DIM, K>(M1s, u, t, y, nel);  // ends with __syncthreads
      for (int w = threadIdx.x; w < items; w += NTT)
        ke += rho0K[el0 + w / (DIM * ND1)] * vc[w] * y[w];
      __syncthreads();
    }
    for (int64_t el = threadIdx.x; el < g.nelem; el += NTT) {
      double s = 0.0;
      for (int j = 0; j < ND2; ++j) s += bas.L2int[j] * e[el * ND2 + j];
      ie += rho0K[el] * s;
    }
    const double tot = cta_sum(0.5 * ke + ie);
    if (threadIdx.x == 0) a.out[i] = tot;
  }
}

// Kernels of one launch shape (threads per CTA, points per thread) and their
// shared memory.
struct BOps {
  int ntt, qpt;
  size_t (*stage_bytes)(int64_t nnodes_max, int smem_lines);
  size_t energy_bytes;
  const void* stage;
  const void* estimate;
  const void* sampled;
  const void* energy;
};

template <int DIM, int K, bool MIXED, int NTT, int QPT = 1>
static BOps make_batch_ops() {
  using L = BL<DIM, K, MIXED, NTT, QPT>;
  BOps o;
  o.ntt = NTT;
  o.qpt = QPT;
  o.stage_bytes = &L::bytes;
  constexpr int P = K + 1, ND1 = ipow(P, DIM);
  o.energy_bytes = (size_t)(4 * L::CGT * DIM * ND1 + P * P) * sizeof(double);
  o.stage = (const void*)batch_stage_kernel<DIM, K, MIXED, NTT, QPT>;
  o.estimate = (const void*)batch_estimate_kernel<DIM, K, MIXED, NTT>;
  o.sampled = (const void*)batch_sampled_kernel<DIM, K, MIXED, NTT>;
  o.energy = (const void*)batch_energy_kernel<DIM, K, NTT>;
  return o;
}

// Instantiated in batch_2d.cu / batch_3d.cu (one translation unit per
// dimension, so they compile in parallel).  False if the shape is not built.
bool get_batch_ops_2d_q1(int k, bool mixed, int ntt, int qpt, BOps* out);
bool get_batch_ops_2d_q2(int k, bool mixed, int ntt, int qpt, BOps* out);
bool get_batch_ops_3d(int k, bool mixed, int ntt, int qpt, BOps* out);

}  // namespace lagh
