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
//  - tensor product: with rho0|J0| the same in every element, M_V restricted
//    to the free entries of component c is rho0|J0| times the Kronecker
//    product of assembled 1D reference mass matrices G_d (without their end
//    nodes along direction c).  The inverse of each G_d decays exponentially
//    away from the diagonal; its entries within a band of half-width B are
//    kept in FP32 and applied by one line pass per direction (a tile of node
//    lines and its halo staged in shared memory).  The CG converges in about
//    three iterations (Jacobi needs ~28 on the 64x64 Taylor-Green mesh).  On
//    narrow meshes (the 2D tile kernel, the narrow line passes, the cluster
//    solve) of the mixed path, each band entry is the FP32 pair hi + lo of
//    its FP64 value and every sum is formed without rounding error (exact
//    products, TwoSum, the errors collected apart): the preconditioner is then
//    accurate to the FP32 rounding of its input, and the CG converges in two
//    iterations.  The FP64 path keeps the plain FP32 sums and three
//    iterations, which take its solves far below the tolerance: it is held to
//    1e-8 of the oracle after tens of thousands of steps, where the solves'
//    own errors (up to cond(M_V) times the tolerance) add up;
//  - Jacobi: the inverse assembled diagonal.
#include <cooperative_groups.h>

#include "line_solve.cuh"
#include "mass_ops.cuh"

namespace lagh {

constexpr int kLineThreads = 256;  // one CTA per tile of LT node lines x 32 positions
// band half-width of the truncated 1D inverses, by H1 order (must match setup)
template <int K> struct PB { static constexpr int B = K == 1 ? 14 : (K == 2 ? 22 : 30); };
constexpr int kNodeThreads = 256;
enum { kTicketPass0 = 0, kTicketPassL = 1, kTicketA = 2, kTicketB = 3, kTicketJ = 4 };

struct CgArgs {
  Geom g;
  double M1[(kMaxOrder + 1) * (kMaxOrder + 1)];
  TensorPC tpc;
  const float* lfac;
  const float* lfac_lo;
  const double* lfac64;
  const double* lchol;
  const double* rhs;
  double *x, *r, *z, *p, *Ap, *ApE;
  double* r2;            // second residual buffer of the 2D tile kernel
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
  int standalone;        // a preconditioner application outside a solve: never gated
  int comp;              // narrow band passes with error-free sums (mixed path)
};

__device__ __forceinline__ bool gated(const CgArgs& a) {
  return !a.standalone && ((a.gate != nullptr && a.gate->done) || a.cg->done);
}

// Sum of the per-block partials by the whole (last) block, in a fixed order:
// thread t adds partials t, t + blockDim, ... in sequence, then a fixed tree.
// All threads must call it; the result is valid in thread 0.
__device__ __forceinline__ double sum_partials(const double* part) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (unsigned int i = threadIdx.x; i < gridDim.x; i += blockDim.x) acc += __ldcg(&part[i]);
  return block_sum(acc, sh);
}

// The ticket of a finished block: one GPU-scope acquire-release increment.
// Its release publishes the partials this thread stored before it; for the
// last block its acquire, carried to the block's other threads by the
// following barrier, makes every other block's partials visible.
__device__ __forceinline__ unsigned int take_ticket(unsigned int* ticket) {
  unsigned int old;
  asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(old) : "l"(ticket) : "memory");
  return old;
}

// Block partial -> the last block to finish adds all partials (sum_partials).
// Returns true in every thread of the last block; *total is valid in thread 0.
__device__ __forceinline__ bool reduce_last(double v, double* part, unsigned int* ticket,
                                            double* total) {
  __shared__ double sh[32];
  __shared__ bool last;
  double s = block_sum(v, sh);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = s;
    last = (take_ticket(ticket) == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return false;
  const double tot = sum_partials(part);
  if (threadIdx.x == 0) {
    *total = tot;
    *ticket = 0u;
  }
  __syncthreads();
  return true;
}

// Block partial only (the caller's last block reads it back); thread 0 then
// takes its ticket in reduce_last, whose release publishes this store too.
__device__ __forceinline__ void write_partial(double v, double* part) {
  __shared__ double sh[32];
  double s = block_sum(v, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__device__ __forceinline__ void report(const CgArgs& a, bool conv, double rr) {
  CgDev* cg = a.cg;
  a.ctl->cg_last_iters = cg->it;
  a.ctl->cg_last_relres = cg->bb > 0.0 ? sqrt(rr / cg->bb) : 0.0;
  a.ctl->cg_iters += cg->it;
  if (!conv) atomicOr(&a.ctl->status, kDevCG);
}

// The end of CG iteration it (thread 0 of the last block of the kernel that
// completed |r|^2): counts the iteration and applies the convergence test
// |r| <= rtol |b|, a NaN guard and the iteration cap; a finished solve sets
// done, reports, and ends the WHILE loop.  Returns true if it finished.
__device__ __forceinline__ bool end_iteration(const CgArgs& a, double rr) {
  CgDev* cg = a.cg;
  cg->it += 1;
  const bool conv = rr <= a.rtol * a.rtol * cg->bb;
  const bool bad = !(rr == rr);
  if (conv || bad || cg->it >= a.maxit) {
    cg->done = 1;
    report(a, conv, rr);
    if (a.has_cond) cudaGraphSetConditional(a.cond, 0);
    return true;
  }
  return false;
}

// ---------------------------------------------------- tensor line passes --

// One pass of the tensor-product preconditioner along direction d: every
// node line of every component is multiplied by the banded inverse of the 1D
// mass matrix.  A CTA owns a tile of LT (8 or 32) node lines x 32 positions:
// it stages the tile and its +-B halo along the line in shared memory
// (coalesced: along x the lines are contiguous rows, along y / z neighbouring
// lines are neighbouring nodes), then each of its 256 threads forms LT / 8
// outputs in FP32.
//
// mode: 0 = first pass of the initial preconditioning (reads rhs, writes r = b
// on free components and x = 0, sums b.b), 1 = first pass inside the loop
// (reads r), 2 = later pass (reads z, writes z2 / z alternately, see caller).
// last: the pass along the last direction (sums r.z; init also writes p = z).
// Shared memory of one band-pass tile: LT lines x (32 positions + halo) of
// input, the band rows of the 32 positions in the band's precision T, and the
// first entry and kind of each of the tile's lines.
template <int K, typename T = float, int LTV = 32>
struct PassTile {
  static constexpr int B = PB<K>::B, W = 2 * B + 1, TP = 32, ldt = TP + 2 * B + 1;
  static constexpr int LT = LTV;  // node lines per tile
  // narrow FP32 passes: error-free sums with the band's low parts (band_fma)
  static constexpr bool COMP = sizeof(T) == 4 && LTV == 8;
  T tile[LT * ldt];
  T wrows[TP * W];
  float wlo[COMP ? TP * W : 1];
  int64_t lbase[LT];  // first entry of each tile line
  int lflag[LT];      // 0: past the last line, 1: free line, 2: wall-normal line (all zero)
};

// S + C += (wh + wl) t without rounding error in the main term: the product
// wh t split exactly into p + pe (FMA), wl t rounded, p added to S by TwoSum
// and every error collected in C.
__device__ __forceinline__ void band_fma(float wh, float wl, float t, float& S, float& C) {
  const float p = __fmul_rn(wh, t);
  const float pe = __fmaf_rn(wh, t, -p);
  float s2, e2;
  two_sum_f(S, p, s2, e2);
  S = s2;
  C = __fadd_rn(C, __fadd_rn(e2, __fmaf_rn(wl, t, pe)));
}

template <int DIM>
__host__ __device__ __forceinline__ int64_t pass_tiles(const Geom& g, int d, int lt) {
  const int nd = g.nn[d];
  const int64_t nlines = g.nnodes / nd;
  return (int64_t)DIM * ((nlines + lt - 1) / lt) * ((nd + 31) / 32);
}

// One tile of a band pass along direction d (all threads of the block): the
// tile's outputs dst = band-inverse(src) and, per mode, r / x / p writes and
// the partial sums b.b (mode 0) and r.z (last), added to l_bb / l_rz.
//
// upd (loop passes of the band preconditioner) fuses the CG update with the
// passes: 1 = first pass, stages r - alpha Ap instead of r, adds alpha p to x
// at its outputs and sums |r - alpha Ap|^2 into l_rr; 2 = last pass, stores
// r - alpha Ap at its outputs and takes r.z with it.  Both sides form the
// new residual with the same fused multiply-add, so they agree bitwise.
template <int DIM, int K, typename T = float, int LTV = 32>
__device__ __forceinline__ void pass_tile(const CgArgs& a, int d, int mode, int last, int init,
                                          const double* src_in, double* dst, int64_t bid,
                                          PassTile<K, T, LTV>& sm, double& l_bb, double& l_rz,
                                          int upd = 0, double alpha = 0.0,
                                          double* l_rr = nullptr) {
  using PT = PassTile<K, T, LTV>;
  constexpr int B = PT::B, W = PT::W, TP = PT::TP, ldt = PT::ldt, LT = PT::LT;
  T* tile = sm.tile;
  T* wrows = sm.wrows;
  const Geom& g = a.g;
  const int nd = g.nn[d];
  const int64_t nlines = g.nnodes / nd;
  const int64_t lgroups = (nlines + LT - 1) / LT;
  const int pblocks = (nd + TP - 1) / TP;
  const int64_t stride = d == 0 ? 1 : (d == 1 ? (int64_t)g.nn[0] : (int64_t)g.nn[0] * g.nn[1]);
  // tile -> (component, line group, position block)
  const int pb = (int)(bid % pblocks);
  bid /= pblocks;
  const int64_t lg = bid % lgroups;
  const int c = (int)(bid / lgroups);
  const int p0 = pb * TP;
  const int var = (c == d) ? 1 : 0;
  const int tid = threadIdx.x, nt = blockDim.x;
  // line l of the tile: its base node and whether it is a wall-normal line
  auto line_info = [&](int l, int64_t& base, bool& wall) -> bool {
    const int64_t line = lg * LT + l;
    if (line >= nlines) return false;
    int I[3] = {0, 0, 0};
    if (d == 0) { I[1] = (int)(line % g.nn[1]); I[2] = (int)(line / g.nn[1]); }
    else if (d == 1) { I[0] = (int)(line % g.nn[0]); I[2] = (int)(line / g.nn[0]); }
    else { I[0] = (int)(line % g.nn[0]); I[1] = (int)(line / g.nn[0]); }
    base = (int64_t)c * g.nnodes + node_index(g, I[0], I[1], I[2]);
    wall = (c != d) && (I[c] == 0 || I[c] == g.nn[c] - 1);
    return true;
  };
  const double* src = mode == 0 ? a.rhs : src_in;
  const T scl = (mode == 2) ? T(1) : (T)a.tpc.scale;
  // the tile's lines, once (their 64-bit index arithmetic stays out of the loops)
  for (int l = tid; l < LT; l += nt) {
    int64_t base = 0;
    bool wall = false;
    const bool ok = line_info(l, base, wall);
    sm.lbase[l] = base;
    sm.lflag[l] = ok ? (wall ? 2 : 1) : 0;
  }
  __syncthreads();
  // stage the tile with its halo: positions [p0 - B, p0 + TP + B); each thread
  // issues its loads CH at a time into registers before it stores them (one
  // guarded load per iteration behind the previous store runs them serially)
  constexpr int span = TP + 2 * B, CH = 4;
  for (int i0 = tid; i0 < LT * span; i0 += CH * nt) {
    double v[CH];
    bool ok[CH];
#pragma unroll
    for (int j = 0; j < CH; ++j) {
      const int idx = i0 + j * nt;
      // along x (d == 0) walk a line, otherwise walk across lines
      const int l = d == 0 ? idx / span : idx % LT;
      const int q = d == 0 ? idx - l * span : idx / LT;
      const int pos = p0 - B + q;
      ok[j] = idx < LT * span && pos >= var && pos < nd - var && sm.lflag[l] == 1;
      const int64_t k = ok[j] ? sm.lbase[l] + pos * stride : 0;
      v[j] = ok[j] ? src[k] : 0.0;
      if (upd == 1 && ok[j]) v[j] = fma(-alpha, a.Ap[k], v[j]);
    }
#pragma unroll
    for (int j = 0; j < CH; ++j) {
      const int idx = i0 + j * nt;
      if (idx < LT * span) {
        const int l = d == 0 ? idx / span : idx % LT;
        const int q = d == 0 ? idx - l * span : idx / LT;
        tile[l * ldt + q] = ok[j] ? (T)v[j] * scl : T(0);
      }
    }
  }
  {
    const int nrow = nd - 2 * var;  // rows of the band (interior positions)
    for (int idx = tid; idx < TP * W; idx += nt) {
      const int q = idx / W, m = idx - q * W;
      const int row = p0 + q - var;
      T wv = T(0);
      float wl = 0.0f;
      if (row >= 0 && row < nrow) {
        if constexpr (sizeof(T) == 8) {
          wv = a.lfac64[a.tpc.off64[d][var] + (int64_t)row * W + m];
        } else {
          wv = a.lfac[a.tpc.off[d][var] + (int64_t)row * W + m];
          if constexpr (PT::COMP)
            if (a.comp) wl = a.lfac_lo[a.tpc.off[d][var] + (int64_t)row * W + m];
        }
      }
      wrows[idx] = wv;
      if constexpr (PT::COMP) sm.wlo[idx] = wl;
      (void)wl;
    }
  }
  __syncthreads();
  for (int o = tid; o < LT * TP; o += nt) {
    const int l = d == 0 ? o / TP : o % LT;
    const int q = d == 0 ? o - l * TP : o / LT;
    const int pos = p0 + q;
    const int fl = sm.lflag[l];
    if (pos >= nd || fl == 0) continue;
    const bool wall = fl == 2;
    const int64_t kk = sm.lbase[l] + pos * stride;
    double zv = 0.0;
    if (!wall && pos >= var && pos < nd - var) {
      const T* wr = wrows + q * W;
      const T* tr = tile + l * ldt + q;  // tile position of offset -B
      bool done = false;
      if constexpr (PT::COMP) {
        if (a.comp) {
        // error-free sum; the last pass widens S + C to FP64, an inner pass
        // rounds it to FP32 (the next pass stages FP32 values)
        const float* wlr = sm.wlo + q * W;
        float S = 0.0f, C = 0.0f;
#pragma unroll
        for (int m = 0; m < W; ++m) band_fma(wr[m], wlr[m], tr[m], S, C);
        zv = last ? f2d_exact(S) + f2d_exact(C) : (double)__fadd_rn(S, C);
        done = true;
        }
      }
      if (!done) {
        T acc = T(0);
#pragma unroll
        for (int m = 0; m < W; ++m) {
          if constexpr (sizeof(T) == 4) acc = __fmaf_rn(wr[m], tr[m], acc);
          else acc = fma(wr[m], tr[m], acc);
        }
        zv = (double)acc;
      }
    }
    if (mode == 0) {
      const bool ess = wall || pos < var || pos >= nd - var;
      const double bv = ess ? 0.0 : a.rhs[kk];
      a.r[kk] = bv;
      a.x[kk] = 0.0;
      l_bb += bv * bv;
    }
    if (upd == 1) {
      const double rv = fma(-alpha, a.Ap[kk], a.r[kk]);
      a.x[kk] = fma(alpha, a.p[kk], a.x[kk]);
      *l_rr += rv * rv;
    }
    dst[kk] = zv;
    if (last) {
      double rv = a.r[kk];
      if (upd == 2) {
        rv = fma(-alpha, a.Ap[kk], rv);
        a.r[kk] = rv;
      }
      l_rz += rv * zv;
      if (init) a.p[kk] = zv;
    }
  }
  __syncthreads();  // the tile buffers are reused by the next tile
}

// One pass of the tensor-product preconditioner along direction d over one
// tile per CTA (pass_tile), at most 4 CTAs of 256 threads per SM (64
// registers).
//
// mode: 0 = first pass of the initial preconditioning (reads rhs, writes r = b
// on free components and x = 0, sums b.b), 1 = first pass inside the loop
// (reads r), 2 = later pass (reads z, writes z2 / z alternately, see caller).
// last: the pass along the last direction (sums r.z; init also writes p = z).
// upd: the CG update fused into the loop passes (see pass_tile); the first
// pass ends the iteration with the convergence test on |r|^2.
template <int DIM, int K, typename T, int LTV>
__global__ void __launch_bounds__(kLineThreads, 4) cg_pass_kernel(const CgArgs a, int d, int mode,
                                                              int last, int init, int upd,
                                                              const double* src_in,
                                                              double* dst) {
  pdl_enter();
  if (init ? (a.gate != nullptr && a.gate->done) : gated(a)) {
    if (upd == 1 && a.has_cond && blockIdx.x == 0 && threadIdx.x == 0)
      cudaGraphSetConditional(a.cond, 0);
    return;
  }
  if (mode == 0 && blockIdx.x == 0 && threadIdx.x == 0) {  // a new solve
    a.cg->done = 0;
    a.cg->it = 0;
  }
  __shared__ PassTile<K, T, LTV> sm;
  double l_bb = 0.0, l_rz = 0.0, l_rr = 0.0;
  const double alpha = upd != 0 ? a.cg->alpha : 0.0;
  pass_tile<DIM, K, T, LTV>(a, d, mode, last, init, src_in, dst, (int64_t)blockIdx.x, sm, l_bb,
                            l_rz, upd, alpha, &l_rr);
  double tot;
  if (upd == 1) {
    if (reduce_last(l_rr, a.part + 4 * kMaxPartials, &a.cg->ticket[kTicketB], &tot) &&
        threadIdx.x == 0)
      end_iteration(a, tot);
  }
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
        cg->beta = 0.0;
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

// ------------------------------------------------ 2D fused band passes ----

// Both directions of the 2D band preconditioner in one kernel, for meshes
// whose line passes would leave SMs idle.  A CTA owns a tile of the nodes of
// one component: 16 x 16, where a last tile along a direction takes the
// remaining node lines (1 to 16; a single remaining line, as for any mesh of
// 16m elements per direction, joins the tile before it, 17 wide).  It stages
// the input over the tile and a +-B window in both directions, applies the x
// band to every window row at the tile's columns, then the y band to that.
// Each output is the same sum of the same products, in the same order, as
// the narrow x pass followed by the y pass (plain FP32, or error-free with
// band_fma on the mixed path, the x result rounded once to FP32), so the
// result is bitwise that of the two line passes (which widen the rounded x
// result to FP64 and back, exactly).
//
// mode / init / upd as for cg_pass_kernel, with both passes in this one
// (first and last): mode 0 initial (b.b and r.z), upd 1 the CG update fused
// (r.z and |r|^2, then the convergence test), otherwise a plain application
// (r.z).  With the update fused, a CTA stages r - alpha Ap over its halo while
// other CTAs form the new residual of their own nodes, so the residual
// alternates between two buffers by iteration parity: iteration it (counted
// from 0) reads r[it & 1] and writes r[(it + 1) & 1]; the initial application
// writes r[0].
template <int K>
struct Pass2DTile {
  static constexpr int B = PB<K>::B, W = 2 * B + 1, TS = 16, TM = TS + 1, WN = TM + 2 * B;
  static constexpr int ldw = ((WN + 15) / 32) * 32 + 16;  // row stride = 16 (mod 32) banks
  float win[WN * ldw];   // input window [y][x], positions y0 - B.., x0 - B..
  float tx[WN * TM];     // x-band result on the window rows at the tile columns
  float wxT[W * TM];     // x band rows of the tile columns, [m][column]
  float wy[TM * W];      // y band rows of the tile rows, [row][m]
  float wxTl[W * TM];    // their low parts (band_fma)
  float wyl[TM * W];
};

// Tiles along a line of n nodes: 16 wide, the last one ragged or 17 wide.
__host__ __device__ __forceinline__ int pass2d_tiles(int n) {
  const int t = (n + 15) / 16;
  return (n % 16 == 1 && t > 1) ? t - 1 : t;
}

template <int K>
__global__ void __launch_bounds__(kLineThreads) cg_pass2d_kernel(const CgArgs a, int mode,
                                                                int init, int upd,
                                                                double* dst) {
  using PT = Pass2DTile<K>;
  constexpr int B = PT::B, W = PT::W, TS = PT::TS, TM = PT::TM, WN = PT::WN, ldw = PT::ldw;
  constexpr int NT = kLineThreads;
  pdl_enter();
  if (init ? (a.gate != nullptr && a.gate->done) : gated(a)) {
    if (upd == 1 && a.has_cond && blockIdx.x == 0 && threadIdx.x == 0)
      cudaGraphSetConditional(a.cond, 0);
    return;
  }
  if (mode == 0 && blockIdx.x == 0 && threadIdx.x == 0) {  // a new solve
    a.cg->done = 0;
    a.cg->it = 0;
  }
  __shared__ PT sm;
  const Geom& g = a.g;
  const int n0 = g.nn[0], n1 = g.nn[1];
  const int ntx = pass2d_tiles(n0), nty = pass2d_tiles(n1);
  const int tile = (int)(blockIdx.x % (unsigned)(ntx * nty));
  const int c = (int)(blockIdx.x / (unsigned)(ntx * nty));
  const int tix = tile % ntx, tiy = tile / ntx;
  const int x0 = tix * TS, y0 = tiy * TS;
  const int wx = tix == ntx - 1 ? n0 - x0 : TS, wy = tiy == nty - 1 ? n1 - y0 : TS;  // <= TM
  const int wnx = wx + 2 * B, wny = wy + 2 * B;  // window extent, <= WN
  const int tid = threadIdx.x;
  const int64_t cbase = (int64_t)c * g.nnodes;
  // free nodes of component c: the end nodes along direction c are essential
  auto is_free = [&](int x, int y) -> bool {
    if (x < 0 || x >= n0 || y < 0 || y >= n1) return false;
    return c == 0 ? (x > 0 && x < n0 - 1) : (y > 0 && y < n1 - 1);
  };
  const int it0 = upd == 1 ? a.cg->it : 0;  // iterations completed before this one
  const double* rin = upd == 1 ? ((it0 & 1) ? a.r2 : a.r) : a.r;
  double* rout = (upd == 1 && !(it0 & 1)) ? a.r2 : a.r;
  const double* src = mode == 0 ? a.rhs : rin;
  const float scl = (float)a.tpc.scale;
  const double alpha = upd != 0 ? a.cg->alpha : 0.0;
  // Every global load is issued before the shared-memory stores that would
  // otherwise order it (a guarded load per loop iteration ran the loads one
  // after another: 2.4 us more per launch for the window alone).  First the
  // band rows (direction d's rows exclude the end nodes when d == c) and the
  // operands of this thread's outputs, then the window in batches of 8.
  constexpr int PB_ = (TM * W + NT - 1) / NT, PO = (TM * TM + NT - 1) / NT;
  const int vx = (c == 0) ? 1 : 0, vy = (c == 1) ? 1 : 0;
  float bxv[PB_], byv[PB_], bxl[PB_], byl[PB_];
  {
    const int64_t ox = a.tpc.off[0][vx], oy = a.tpc.off[1][vy];
#pragma unroll
    for (int j = 0; j < PB_; ++j) {
      const int idx = tid + j * NT;
      const int qq = idx / W, m = idx - qq * W;
      const int rx = x0 + qq - vx, ry = y0 + qq - vy;
      const bool inb = idx < TM * W;
      const bool okx = inb && qq < wx && rx >= 0 && rx < n0 - 2 * vx;
      const bool oky = inb && qq < wy && ry >= 0 && ry < n1 - 2 * vy;
      const int64_t kx = ox + (int64_t)rx * W + m, ky = oy + (int64_t)ry * W + m;
      bxv[j] = okx ? a.lfac[kx] : 0.0f;
      bxl[j] = (okx && a.comp) ? a.lfac_lo[kx] : 0.0f;
      byv[j] = oky ? a.lfac[ky] : 0.0f;
      byl[j] = (oky && a.comp) ? a.lfac_lo[ky] : 0.0f;
    }
  }
  double o_r[PO], o_ap[PO], o_p[PO], o_x[PO];
#pragma unroll
  for (int j = 0; j < PO; ++j) {
    const int o = tid + j * NT;  // this tile's wy x wx nodes, row by row
    const int yl = o / wx, q = o - yl * wx;
    const bool own = o < wx * wy;
    const int x = x0 + q, y = y0 + yl;
    const int64_t kk = own ? cbase + (int64_t)y * n0 + x : 0;
    o_r[j] = o_ap[j] = o_p[j] = o_x[j] = 0.0;
    if (own) {
      if (mode == 0) {
        o_r[j] = is_free(x, y) ? a.rhs[kk] : 0.0;
      } else {
        o_r[j] = rin[kk];
        if (upd == 1) {
          o_ap[j] = a.Ap[kk];
          o_p[j] = a.p[kk];
          o_x[j] = a.x[kk];
        }
      }
    }
  }
  {
    constexpr int PER = (WN * WN + NT - 1) / NT;
    constexpr int CH = 8;
#pragma unroll
    for (int c0 = 0; c0 < PER; c0 += CH) {
      double v[CH];
      bool ok[CH];
#pragma unroll
      for (int j = 0; j < CH; ++j) {
        const int idx = tid + (c0 + j) * NT;
        const int wyi = idx / WN, wxi = idx - wyi * WN;
        const int x = x0 - B + wxi, y = y0 - B + wyi;
        ok[j] = idx < WN * WN && wxi < wnx && wyi < wny && is_free(x, y);
        const int64_t k = cbase + (int64_t)(ok[j] ? y : 0) * n0 + (ok[j] ? x : 0);
        v[j] = ok[j] ? src[k] : 0.0;
        if (upd == 1 && ok[j]) v[j] = fma(-alpha, a.Ap[k], v[j]);
      }
#pragma unroll
      for (int j = 0; j < CH; ++j) {
        const int idx = tid + (c0 + j) * NT;
        if (idx < WN * WN) {
          const int wyi = idx / WN, wxi = idx - wyi * WN;
          sm.win[wyi * ldw + wxi] = ok[j] ? (float)v[j] * scl : 0.0f;
        }
      }
    }
  }
#pragma unroll
  for (int j = 0; j < PB_; ++j) {
    const int idx = tid + j * NT;
    if (idx < TM * W) {
      const int qq = idx / W, m = idx - qq * W;
      sm.wxT[m * TM + qq] = bxv[j];
      sm.wy[idx] = byv[j];
      sm.wxTl[m * TM + qq] = bxl[j];
      sm.wyl[idx] = byl[j];
    }
  }
  __syncthreads();
  // x band on the window rows, tile columns (zero off the free set)
  // (the wny x wx entries the y band reads, spread evenly over the threads)
  for (int o = tid; o < wny * wx; o += NT) {
    const int wyi = o / wx, qq = o - wyi * wx;
    float S = 0.0f, C = 0.0f;
    if (is_free(x0 + qq, y0 - B + wyi)) {
      const float* wr = sm.win + wyi * ldw + qq;
      if (a.comp) {
#pragma unroll
        for (int m = 0; m < W; ++m) band_fma(sm.wxT[m * TM + qq], sm.wxTl[m * TM + qq], wr[m], S, C);
      } else {
#pragma unroll
        for (int m = 0; m < W; ++m) S = __fmaf_rn(sm.wxT[m * TM + qq], wr[m], S);
      }
    }
    sm.tx[wyi * TM + qq] = a.comp ? __fadd_rn(S, C) : S;
  }
  __syncthreads();
  double l_bb = 0.0, l_rz = 0.0, l_rr = 0.0;
#pragma unroll
  for (int j = 0; j < PO; ++j) {
    const int o = tid + j * NT;
    const int yl = o / wx, q = o - yl * wx;
    if (o >= wx * wy) continue;
    const int x = x0 + q, y = y0 + yl;
    const int64_t kk = cbase + (int64_t)y * n0 + x;
    const bool fr = is_free(x, y);
    double zv = 0.0;
    if (fr) {
      const float* tr = sm.tx + yl * TM + q;  // window row y - B
      const float* wr = sm.wy + yl * W;
      const float* wl = sm.wyl + yl * W;
      float S = 0.0f, C = 0.0f;
      if (a.comp) {
#pragma unroll
        for (int m = 0; m < W; ++m) band_fma(wr[m], wl[m], tr[m * TM], S, C);
        zv = f2d_exact(S) + f2d_exact(C);
      } else {
#pragma unroll
        for (int m = 0; m < W; ++m) S = __fmaf_rn(wr[m], tr[m * TM], S);
        zv = (double)S;
      }
    }
    double rv = o_r[j];
    if (mode == 0) {
      a.x[kk] = 0.0;
      l_bb += rv * rv;
      rout[kk] = rv;
    } else if (upd == 1) {
      rv = fma(-alpha, o_ap[j], o_r[j]);
      a.x[kk] = fma(alpha, o_p[j], o_x[j]);
      l_rr += rv * rv;
      rout[kk] = rv;
    }
    dst[kk] = zv;
    l_rz += rv * zv;
    if (init) a.p[kk] = zv;
  }
  double tot;
  if (mode == 0) {
    write_partial(l_bb, a.part);
    if (reduce_last(l_rz, a.part + kMaxPartials, &a.cg->ticket[kTicketPassL], &tot)) {
      const double bb = sum_partials(a.part);
      if (threadIdx.x != 0) return;
      CgDev* cg = a.cg;
      cg->bb = bb;
      cg->rz = tot;
      cg->it = 0;
      cg->beta = 0.0;
      if (!(bb > 0.0)) {  // zero right-hand side: x = 0 is the solution
        cg->done = 1;
        report(a, true, 0.0);
      }
    }
  } else if (upd == 1) {
    // every block writes its r.z partial before it takes its |r|^2 ticket
    write_partial(l_rz, a.part + 3 * kMaxPartials);
    if (reduce_last(l_rr, a.part + 4 * kMaxPartials, &a.cg->ticket[kTicketB], &tot)) {
      const double rz_new = sum_partials(a.part + 3 * kMaxPartials);
      if (threadIdx.x != 0) return;
      CgDev* cg = a.cg;
      if (!end_iteration(a, tot)) {
        cg->beta = rz_new / cg->rz;
        cg->rz = rz_new;
      }
    }
  } else {
    if (reduce_last(l_rz, a.part + kMaxPartials, &a.cg->ticket[kTicketPassL], &tot) &&
        threadIdx.x == 0) {
      a.cg->beta = tot / a.cg->rz;
      a.cg->rz = tot;
    }
  }
}

// ------------------------------------------------- exact line solves ----

// One direction of the exact tensor-product preconditioner: every node line
// of every component along direction d is solved with the banded Cholesky
// factor of its assembled 1D matrix (forward and backward substitution,
// FP64).  A CTA owns kLineGroup lines of one component: it stages them in
// shared memory (coalesced), kLineGroup threads solve one line each, and the
// block writes them back.  mode / last / init as for cg_pass_kernel.
constexpr int kLineGroup = 8;
constexpr int kLineThreadsX = 64;

template <int DIM, int K>
__global__ void __launch_bounds__(kLineThreadsX) cg_line_kernel(const CgArgs a, int d, int mode,
                                                               int last, int init,
                                                               const double* src_in,
                                                               double* dst) {
  pdl_enter();
  if (init ? (a.gate != nullptr && a.gate->done) : gated(a)) return;
  if (mode == 0 && blockIdx.x == 0 && threadIdx.x == 0) {  // a new solve
    a.cg->done = 0;
    a.cg->it = 0;
  }
  extern __shared__ double lbuf[];
  const Geom& g = a.g;
  const int nd = g.nn[d];
  const int ldb = nd | 1;  // odd row length (bank spread)
  const int64_t nlines = g.nnodes / nd;
  const int64_t groups = (nlines + kLineGroup - 1) / kLineGroup;
  const int c = (int)(blockIdx.x / groups);
  const int64_t l0 = (int64_t)(blockIdx.x % groups) * kLineGroup;
  const int var = (c == d) ? 1 : 0;
  const int64_t stride = d == 0 ? 1 : (d == 1 ? (int64_t)g.nn[0] : (int64_t)g.nn[0] * g.nn[1]);
  const int tid = threadIdx.x;
  // line l of the group: its first node and whether it is a wall-normal line
  auto line_info = [&](int l, int64_t& base, bool& wall) -> bool {
    const int64_t line = l0 + l;
    if (line >= nlines) return false;
    int I[3] = {0, 0, 0};
    if (d == 0) { I[1] = (int)(line % g.nn[1]); I[2] = (int)(line / g.nn[1]); }
    else if (d == 1) { I[0] = (int)(line % g.nn[0]); I[2] = (int)(line / g.nn[0]); }
    else { I[0] = (int)(line % g.nn[0]); I[1] = (int)(line / g.nn[0]); }
    base = (int64_t)c * g.nnodes + node_index(g, I[0], I[1], I[2]);
    wall = (c != d) && (I[c] == 0 || I[c] == g.nn[c] - 1);
    return true;
  };
  const double* src = mode == 0 ? a.rhs : src_in;
  const double scl = (mode == 2) ? 1.0 : a.tpc.scale;
  // along x the lines are rows (walk a line), otherwise neighbouring lines
  // are neighbouring nodes (walk across lines)
  for (int idx = tid; idx < kLineGroup * nd; idx += kLineThreadsX) {
    const int l = d == 0 ? idx / nd : idx % kLineGroup;
    const int pos = d == 0 ? idx - l * nd : idx / kLineGroup;
    int64_t base;
    bool wall;
    double val = 0.0;
    if (line_info(l, base, wall) && !wall && pos >= var && pos < nd - var)
      val = src[base + pos * stride] * scl;
    lbuf[l * ldb + pos] = val;
  }
  __syncthreads();
  if (tid < kLineGroup) {
    int64_t base;
    bool wall;
    if (line_info(tid, base, wall) && !wall)
      line_solve<K>(lbuf + tid * ldb + var, 1, nd - 2 * var, a.lchol + a.tpc.coff[d][var]);
  }
  __syncthreads();
  double l_bb = 0.0, l_rz = 0.0;
  for (int idx = tid; idx < kLineGroup * nd; idx += kLineThreadsX) {
    const int l = d == 0 ? idx / nd : idx % kLineGroup;
    const int pos = d == 0 ? idx - l * nd : idx / kLineGroup;
    int64_t base;
    bool wall;
    if (!line_info(l, base, wall)) continue;
    const int64_t kk = base + pos * stride;
    const double zv = lbuf[l * ldb + pos];
    if (mode == 0) {
      const bool ess = wall || pos < var || pos >= nd - var;
      const double bv = ess ? 0.0 : a.rhs[kk];
      a.r[kk] = bv;
      a.x[kk] = 0.0;
      l_bb += bv * bv;
    }
    dst[kk] = zv;
    if (last) {
      l_rz += a.r[kk] * zv;
      if (init) a.p[kk] = zv;
    }
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
        cg->beta = 0.0;
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

// ------------------------------------------------ cluster-resident CG ----

// The whole solve of a small problem in one launch: a cluster of CTAs (16
// where the device allows it, else 8) runs the initial preconditioning and
// every iteration, separated by hardware cluster barriers, with the sums
// reduced through distributed shared memory in rank order (every CTA gets the
// same, deterministic value).  Same algorithm and arithmetic as the kernel
// chain (tensor-product band preconditioner, element PA apply, node gather),
// without a launch per phase.
namespace cgx = cooperative_groups;
constexpr int kClusterThreads = 256;

__device__ __forceinline__ double block_sum_all(double v) {
  __shared__ double sh[32];
  __shared__ double res;
  const double s = block_sum(v, sh);
  if (threadIdx.x == 0) res = s;
  __syncthreads();
  return res;
}

// Sum of v over the cluster (every thread of every CTA calls it); slot: this
// reduction's word of shared memory.  Ends with every CTA past a cluster
// barrier, so all global writes made before the call are visible after it.
__device__ __forceinline__ double cluster_sum(cgx::cluster_group& cl, double v, double* slot) {
  const double s = block_sum_all(v);
  if (threadIdx.x == 0) *slot = s;
  cl.sync();
  double tot = 0.0;
  for (unsigned r = 0; r < cl.num_blocks(); ++r) tot += *cl.map_shared_rank(slot, r);
  return tot;
}

// A p element by element (one thread per element and component, the element
// operator in registers): ApE[el][c][i] = rho0K[el] ((M1 x M1) p_K)_i.
template <int K>
__device__ __forceinline__ void elem_apply_2d(const Geom& g, const double* M1s, const double* p,
                                              const double* rho0K, double* ApE, int64_t i0,
                                              int64_t stride) {
  constexpr int P = K + 1, ND1 = P * P;
  for (int64_t item = i0; item < g.nelem * 2; item += stride) {
    const int64_t el = item >> 1;
    const int c = (int)(item & 1);
    int E[3] = {0, 0, 0};
    elem_ijk(g, el, E);
    const double* pc = p + c * g.nnodes;
    double t[P][P];
#pragma unroll
    for (int b = 0; b < P; ++b) {
      double u[P];
#pragma unroll
      for (int a = 0; a < P; ++a) u[a] = pc[elem_node<K>(g, E, a, b, 0)];
#pragma unroll
      for (int ap = 0; ap < P; ++ap) {
        double acc = 0.0;
#pragma unroll
        for (int a = 0; a < P; ++a) acc = fma(M1s[ap * P + a], u[a], acc);
        t[b][ap] = acc;
      }
    }
    const double w = rho0K[el];
    double* out = ApE + (el * 2 + c) * ND1;
#pragma unroll
    for (int bp = 0; bp < P; ++bp)
#pragma unroll
      for (int ap = 0; ap < P; ++ap) {
        double acc = 0.0;
#pragma unroll
        for (int b = 0; b < P; ++b) acc = fma(M1s[bp * P + b], t[b][ap], acc);
        out[bp * P + ap] = w * acc;
      }
  }
}

template <int DIM, int K>
__global__ void __launch_bounds__(kClusterThreads) cg_cluster_kernel(const CgArgs a) {
  pdl_enter();
  if (a.gate != nullptr && a.gate->done) return;  // the same in every CTA
  cgx::cluster_group cl = cgx::this_cluster();
  const int64_t rank = cl.block_rank(), nrank = cl.num_blocks();
  __shared__ PassTile<K, float, 8> sm;
  __shared__ double M1s[(K + 1) * (K + 1)];
  __shared__ double slots[4];
  constexpr int P = K + 1;
  const Geom& g = a.g;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int64_t i0 = rank * nt + tid, stride = nrank * nt;
  for (int i = tid; i < P * P; i += nt) M1s[i] = a.M1[(i / P) * (kMaxOrder + 1) + i % P];
  const int64_t tiles0 = pass_tiles<DIM>(g, 0, 8), tiles1 = pass_tiles<DIM>(g, 1, 8);
  // initial preconditioning: r = b, x = 0, z = B r (x pass into Ap, y pass
  // into z), p = z
  double l_bb = 0.0, l_rz = 0.0;
  for (int64_t t = rank; t < tiles0; t += nrank)
    pass_tile<DIM, K, float, 8>(a, 0, 0, 0, 1, nullptr, a.Ap, t, sm, l_bb, l_rz);
  const double bb = cluster_sum(cl, l_bb, &slots[0]);
  for (int64_t t = rank; t < tiles1; t += nrank)
    pass_tile<DIM, K, float, 8>(a, 1, 2, 1, 1, a.Ap, a.z, t, sm, l_bb, l_rz);
  double rz = cluster_sum(cl, l_rz, &slots[1]);
  int it = 0;
  double rr = bb;
  bool conv = !(bb > 0.0);
  while (!conv && it < a.maxit) {
    ++it;
    elem_apply_2d<K>(g, M1s, a.p, a.rho0K, a.ApE, i0, stride);
    cl.sync();
    double l = 0.0;
    for (int64_t node = i0; node < g.nnodes; node += stride) {
      int I[3];
      node_ijk(g, node, I);
      for (int c = 0; c < DIM; ++c) {
        const int64_t k = c * g.nnodes + node;
        const double ap = essential(g, I, c) ? 0.0 : gather_node<DIM, K>(g, a.ApE, I, c);
        a.Ap[k] = ap;
        l += a.p[k] * ap;
      }
    }
    const double alpha = rz / cluster_sum(cl, l, &slots[2]);
    l = 0.0;
    for (int64_t k = i0; k < g.nv; k += stride) {
      a.x[k] += alpha * a.p[k];
      const double rv = a.r[k] - alpha * a.Ap[k];
      a.r[k] = rv;
      l += rv * rv;
    }
    rr = cluster_sum(cl, l, &slots[3]);
    conv = rr <= a.rtol * a.rtol * bb;
    if (conv || !(rr == rr)) break;
    double unused = 0.0, l_rz2 = 0.0;
    for (int64_t t = rank; t < tiles0; t += nrank)
      pass_tile<DIM, K, float, 8>(a, 0, 1, 0, 0, a.r, a.Ap, t, sm, unused, l_rz2);
    cl.sync();
    for (int64_t t = rank; t < tiles1; t += nrank)
      pass_tile<DIM, K, float, 8>(a, 1, 2, 1, 0, a.Ap, a.z, t, sm, unused, l_rz2);
    const double rz_new = cluster_sum(cl, l_rz2, &slots[0]);
    const double beta = rz_new / rz;
    rz = rz_new;
    for (int64_t k = i0; k < g.nv; k += stride) a.p[k] = a.z[k] + beta * a.p[k];
    cl.sync();
  }
  if (rank == 0 && tid == 0) {
    CgDev* cgd = a.cg;
    cgd->it = it;
    cgd->bb = bb;
    cgd->done = 1;
    a.ctl->cg_last_iters = it;
    a.ctl->cg_last_relres = bb > 0.0 ? sqrt(rr / bb) : 0.0;
    a.ctl->cg_iters += it;
    if (!conv) atomicOr(&a.ctl->status, kDevCG);
  }
  cl.sync();  // no CTA leaves while others may still read its shared memory
}

// ------------------------------------------------------- Jacobi init ----

template <int DIM, int K>
__global__ void __launch_bounds__(kNodeThreads) cg_jacobi_init_kernel(const CgArgs a) {
  pdl_enter();
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
  if (reduce_last(l_rz, a.part + kMaxPartials, &a.cg->ticket[kTicketJ], &rz)) {
    const double bb = sum_partials(a.part);
    if (threadIdx.x != 0) return;
    CgDev* cg = a.cg;
    cg->bb = bb;
    cg->rz = rz;
    cg->it = 0;
    cg->beta = 0.0;
    if (!(cg->bb > 0.0)) {
      cg->done = 1;
      report(a, true, 0.0);
    }
  }
}

// ------------------------------------------------------ loop kernels ----

// Element phase of M p with the search direction formed on the fly,
// p = z + beta p_old (beta = 0 on the first iteration, where p_old = z).
template <int DIM, int K>
__global__ void __launch_bounds__(256) cg_elem_kernel(const CgArgs a) {
  pdl_enter();
  using L = ML<DIM, K>;
  constexpr int P = L::P, ND1 = L::ND1, EPB = L::EPB;
  if (gated(a)) return;
  __shared__ double M1s[P * P];
  __shared__ double u[EPB * DIM * ND1], t[EPB * DIM * ND1], y[EPB * DIM * ND1];
  const Geom& g = a.g;
  for (int i = threadIdx.x; i < P * P; i += blockDim.x) M1s[i] = a.M1[(i / P) * (kMaxOrder + 1) + i % P];
  const double beta = a.cg->beta;
  const int64_t el0 = (int64_t)blockIdx.x * EPB;
  const int nel = (int)((g.nelem - el0) < EPB ? (g.nelem - el0) : EPB);
  const int items = nel * DIM * ND1;
  for (int w = threadIdx.x; w < items; w += blockDim.x) {
    int i = w % ND1, r = w / ND1, c = r % DIM, le = r / DIM;
    int E[3] = {0, 0, 0};
    elem_ijk(g, el0 + le, E);
    int aa = i % P, b = (i / P) % P, cz = DIM == 3 ? i / (P * P) : 0;
    const int64_t k = c * g.nnodes + elem_node<K>(g, E, aa, b, cz);
    u[w] = a.z[k] + beta * a.p[k];
  }
  __syncthreads();
  kron_mass<DIM, K>(M1s, u, t, y, nel);
  for (int w = threadIdx.x; w < items; w += blockDim.x) {
    int le = w / (DIM * ND1);
    a.ApE[el0 * DIM * ND1 + w] = a.rho0K[el0 + le] * y[w];
  }
}

template <int DIM, int K>
__global__ void __launch_bounds__(kNodeThreads) cg_gather_kernel(const CgArgs a) {
  pdl_enter();
  if (gated(a)) return;
  const Geom& g = a.g;
  const double beta = a.cg->beta;
  double l = 0.0;
  for (int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; node < g.nnodes;
       node += (int64_t)gridDim.x * blockDim.x) {
    int I[3];
    node_ijk(g, node, I);
    for (int c = 0; c < DIM; ++c) {
      const int64_t k = c * g.nnodes + node;
      const double ap = essential(g, I, c) ? 0.0 : gather_node<DIM, K>(g, a.ApE, I, c);
      const double pv = a.z[k] + beta * a.p[k];  // the p the element phase used
      a.p[k] = pv;
      a.Ap[k] = ap;
      l += pv * ap;
    }
  }
  double tot;
  if (reduce_last(l, a.part + 2 * kMaxPartials, &a.cg->ticket[kTicketA], &tot) && threadIdx.x == 0)
    a.cg->alpha = a.cg->rz / tot;
}

// x += alpha p, r -= alpha Ap; convergence test; ends the WHILE loop.
template <int DIM, int K>
__global__ void __launch_bounds__(kNodeThreads) cg_update_kernel(const CgArgs a, int jacobi) {
  pdl_enter();
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
  if (reduce_last(l_rr, a.part + 4 * kMaxPartials, &a.cg->ticket[kTicketB], &rr)) {
    // every block wrote its r.z partial before taking its rr ticket
    const double rz_new = jacobi ? sum_partials(a.part + 3 * kMaxPartials) : 0.0;
    if (threadIdx.x != 0) return;
    CgDev* cg = a.cg;
    if (!end_iteration(a, rr) && jacobi) {
      cg->beta = rz_new / cg->rz;
      cg->rz = rz_new;
    }
  }
}

// ------------------------------------------- 2D fused element apply ----

// The element PA apply and the node gather of M p in one kernel, over the
// same 16 x 16 (last 17) node tiles as cg_pass2d_kernel, for the same narrow
// 2D meshes.  A CTA owns the nodes of one tile and one component.  It stages
// p = z + beta p_old over the elements that touch its nodes (the tile's own
// elements and a ring of one element below and to the left, shared with the
// neighbouring tiles), applies rho0K (M1 x M1) to every one of them, and sums
// the element values at its nodes in the gather's element order.  Each
// element product, each rho0K scaling and each node sum is the operation the
// element kernel and the gather kernel perform, in the same order (no fused
// multiply-add across them), so Ap and p are bitwise theirs; only the block
// partials of p.Ap are added over another tiling.
template <int K>
struct Apply2DTile {
  static constexpr int P = K + 1, ND1 = P * P, TS = 16;
  static constexpr int NE1 = (TS + 1 + K - 1) / K + 1;  // elements touching 17 node lines
  static constexpr int NPN = K * NE1 + 1;                // their node lines
  double M1[P * P];
  double r0[NE1 * NE1];     // rho0 |J0| of the patch's elements
  double u[NPN * NPN];      // p = z + beta p_old on the patch of nodes [y][x]
  double t[NE1 * NE1 * ND1];
  double y[NE1 * NE1 * ND1];
};

template <int K>
__global__ void __launch_bounds__(kLineThreads) cg_apply2d_kernel(const CgArgs a) {
  using AT = Apply2DTile<K>;
  constexpr int P = AT::P, ND1 = AT::ND1, TS = AT::TS, NE1 = AT::NE1, NPN = AT::NPN;
  constexpr int NT = kLineThreads;
  pdl_enter();
  if (gated(a)) return;
  __shared__ AT sm;
  const Geom& g = a.g;
  const int n0 = g.nn[0], n1 = g.nn[1];
  const int ntx = pass2d_tiles(n0), nty = pass2d_tiles(n1);
  const int tile = (int)(blockIdx.x % (unsigned)(ntx * nty));
  const int c = (int)(blockIdx.x / (unsigned)(ntx * nty));
  const int tix = tile % ntx, tiy = tile / ntx;
  const int x0 = tix * TS, y0 = tiy * TS;
  const int wx = tix == ntx - 1 ? n0 - x0 : TS, wy = tiy == nty - 1 ? n1 - y0 : TS;
  // elements touching nodes [x0, x0 + wx) x [y0, y0 + wy)
  const int ex0 = x0 > 0 ? (x0 - 1) / K : 0, ey0 = y0 > 0 ? (y0 - 1) / K : 0;
  const int ex1 = min(g.n[0] - 1, (x0 + wx - 1) / K), ey1 = min(g.n[1] - 1, (y0 + wy - 1) / K);
  const int nex = ex1 - ex0 + 1, ney = ey1 - ey0 + 1;  // <= NE1
  const int npx = K * nex + 1, npy = K * ney + 1;       // <= NPN
  const int px0 = K * ex0, py0 = K * ey0;
  const int tid = threadIdx.x;
  const int64_t cbase = (int64_t)c * g.nnodes;
  const double beta = a.cg->beta;
  for (int i = tid; i < P * P; i += NT) sm.M1[i] = a.M1[(i / P) * (kMaxOrder + 1) + i % P];
  {  // the patch's loads all issued before its stores
    constexpr int PER = (NPN * NPN + NT - 1) / NT, PR = (NE1 * NE1 + NT - 1) / NT;
    double zv[PER], pv[PER], rv[PR];
#pragma unroll
    for (int j = 0; j < PR; ++j) {
      const int idx = tid + j * NT;
      const bool ok = idx < nex * ney;
      const int ly = ok ? idx / nex : 0, lx = ok ? idx - ly * nex : 0;
      rv[j] = ok ? a.rho0K[(int64_t)(ex0 + lx) + (int64_t)g.n[0] * (ey0 + ly)] : 0.0;
    }
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      const int idx = tid + j * NT;
      const bool ok = idx < npx * npy;
      const int py = ok ? idx / npx : 0, px = ok ? idx - py * npx : 0;
      const int64_t k = cbase + (int64_t)(py0 + py) * n0 + (px0 + px);
      zv[j] = ok ? a.z[k] : 0.0;
      pv[j] = ok ? a.p[k] : 0.0;
    }
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      const int idx = tid + j * NT;
      if (idx < npx * npy) {
        const int py = idx / npx, px = idx - py * npx;
        sm.u[py * NPN + px] = zv[j] + beta * pv[j];  // as the element kernel forms it
      }
    }
#pragma unroll
    for (int j = 0; j < PR; ++j)
      if (tid + j * NT < nex * ney) sm.r0[tid + j * NT] = rv[j];
  }
  __syncthreads();
  const int items = nex * ney * ND1;
  // contract along x: t[e][b][a'] = sum_a M1[a'][a] u_e[b][a]
  for (int w = tid; w < items; w += NT) {
    const int le = w / ND1, i = w - le * ND1, ap = i % P, b = i / P;
    const int lex = le % nex, ley = le / nex;
    const double* ur = sm.u + (K * ley + b) * NPN + K * lex;
    double s = 0.0;
    for (int aa = 0; aa < P; ++aa) s = fma(sm.M1[ap * P + aa], ur[aa], s);
    sm.t[w] = s;
  }
  __syncthreads();
  // along y: y[e][b'][a] = sum_b M1[b'][b] t[e][b][a]
  for (int w = tid; w < items; w += NT) {
    const int le = w / ND1, i = w - le * ND1, aa = i % P, bp = i / P;
    const double* tr = sm.t + le * ND1 + aa;
    double s = 0.0;
    for (int b = 0; b < P; ++b) s = fma(sm.M1[bp * P + b], tr[b * P], s);
    sm.y[w] = s;
  }
  __syncthreads();
  double l = 0.0;
  for (int o = tid; o < (TS + 1) * (TS + 1); o += NT) {
    const int yl = o / (TS + 1), q = o - yl * (TS + 1);
    if (q >= wx || yl >= wy) continue;
    const int X = x0 + q, Y = y0 + yl;
    // the elements containing the node along x and along y, in increasing
    // order with the node's local index in each (as node_elems_1d)
    const int qx = X / K, rx = X - qx * K, qy = Y / K, ry = Y - qy * K;
    const int fx = (rx == 0 && qx > 0) ? qx - 1 : qx, fy = (ry == 0 && qy > 0) ? qy - 1 : qy;
    const int nx = (rx == 0 && qx > 0 && qx < g.n[0]) ? 2 : 1;
    const int ny = (ry == 0 && qy > 0 && qy < g.n[1]) ? 2 : 1;
    double sacc = 0.0;
#pragma unroll
    for (int ky = 0; ky < 2; ++ky) {
      if (ky >= ny) break;
      const int ey = fy + ky, ly = Y - K * ey;
#pragma unroll
      for (int kx = 0; kx < 2; ++kx) {
        if (kx >= nx) break;
        const int ex = fx + kx, lx = X - K * ex;
        const int le = (ex - ex0) + nex * (ey - ey0);
        sacc = __dadd_rn(sacc, __dmul_rn(sm.r0[le], sm.y[le * ND1 + lx + P * ly]));
      }
    }
    const bool ess = c == 0 ? (X == 0 || X == n0 - 1) : (Y == 0 || Y == n1 - 1);
    const double ap = ess ? 0.0 : sacc;
    const double pv = sm.u[(Y - py0) * NPN + (X - px0)];
    const int64_t k = cbase + (int64_t)Y * n0 + X;
    a.p[k] = pv;
    a.Ap[k] = ap;
    l += pv * ap;
  }
  double tot;
  if (reduce_last(l, a.part + 2 * kMaxPartials, &a.cg->ticket[kTicketA], &tot) && threadIdx.x == 0)
    a.cg->alpha = a.cg->rz / tot;
}

__global__ void cg_reset_kernel(CgDev* cg, const Ctl* gate) {
  pdl_enter();
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
  a.comp = c->precision == LH_MIXED ? 1 : 0;
  a.lfac_lo = c->a.lfac_lo;
  a.lfac64 = c->a.lfac64;
  a.lchol = c->a.lchol;
  a.rhs = rhs;
  a.x = out;
  a.r = c->a.r;
  a.r2 = c->a.r2;
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
  a.standalone = 0;
  return a;
}

static size_t line_smem(const lh_ctx* c, int d) {
  return (size_t)kLineGroup * (c->g.nn[d] | 1) * sizeof(double);
}

// Tiles of 32 node lines where they fill the GPU several times over, else of
// 8 (more CTAs for small meshes; the halo runs along the lines, so shorter
// tiles across the lines cost no extra halo).
template <int DIM>
static bool narrow_passes(const lh_ctx* c) {
  return pass_tiles<DIM>(c->g, 0, 32) < 4 * (int64_t)c->num_sms;
}

// The 2D tile kernels (cg_pass2d_kernel, cg_apply2d_kernel): narrow 2D
// meshes with the FP32 band preconditioner, unless the context turned them off.
template <int DIM>
static bool tiles_2d(const lh_ctx* c) {
  return DIM == 2 && c->cg_tiles && c->tpc.enabled && !c->tpc.exact && !c->tpc.fp64 &&
         narrow_passes<DIM>(c);
}

// Whether the CG update rides on the band passes: where the passes are
// narrow the solve is a chain of latency-bound kernels and one launch fewer
// per iteration pays; on large meshes the separate streaming update is cheaper
// than re-reading Ap with the passes' halos.
template <int DIM>
static bool fuse_update(const lh_ctx* c) {
  return narrow_passes<DIM>(c);
}

// fuse: loop passes of the band preconditioner with the CG update folded in
// (pass_tile's upd); Ap is then still needed by the last pass, so the
// intermediate direction results go to ApE (free after the node gather, and
// at least as long as a velocity vector).
template <int DIM, int K>
static cudaError_t precond_passes(const lh_ctx* c, const CgArgs& a, bool init, cudaStream_t s,
                                  bool fuse = false) {
  // out of place: r -> z (d = 0), then alternate between Ap (free here; ApE
  // when the update is fused) and z so that the last direction writes z; the
  // 2D tile kernel goes from r to z in one launch
  const double* src = a.r;
  double* bufs[2] = {a.z, fuse ? a.ApE : a.Ap};
  if (c->tpc.exact) {
    for (int d = 0; d < DIM; ++d) {
      const int64_t nlines = c->g.nnodes / c->g.nn[d];
      const int64_t blocks = (int64_t)DIM * ((nlines + kLineGroup - 1) / kLineGroup);
      const int mode = d == 0 ? (init ? 0 : 1) : 2;
      double* dst = bufs[(DIM - 1 - d) & 1];
      cudaError_t e = launch_k(c->use_pdl != 0, cg_line_kernel<DIM, K>, dim3((unsigned)blocks),
                               dim3(kLineThreadsX), line_smem(c, d), s, a, d, mode,
                               (int)(d == DIM - 1), init ? 1 : 0, src, dst);
      if (e != cudaSuccess) return e;
      src = dst;
    }
    return cudaGetLastError();
  }
  const bool narrow = narrow_passes<DIM>(c);
  if (tiles_2d<DIM>(c)) {  // both directions in one kernel
    const int64_t blocks = 2 * (int64_t)pass2d_tiles(c->g.nn[0]) * pass2d_tiles(c->g.nn[1]);
    cudaError_t e = launch_k(c->use_pdl != 0, cg_pass2d_kernel<K>, dim3((unsigned)blocks),
                             dim3(kLineThreads), 0, s, a, init ? 0 : 1, init ? 1 : 0,
                             fuse ? 1 : 0, a.z);
    return e != cudaSuccess ? e : cudaGetLastError();
  }
  for (int d = 0; d < DIM; ++d) {
    const int64_t blocks = pass_tiles<DIM>(c->g, d, narrow ? 8 : 32);
    const int mode = d == 0 ? (init ? 0 : 1) : 2;
    double* dst = bufs[(DIM - 1 - d) & 1];
    const bool pdl = c->use_pdl != 0;
    const int last = (int)(d == DIM - 1), ini = init ? 1 : 0;
    const int upd = !fuse ? 0 : (d == 0 ? 1 : (last ? 2 : 0));
    const dim3 gr((unsigned)blocks), bl(kLineThreads);
    cudaError_t e;
    if (c->tpc.fp64)
      e = narrow ? launch_k(pdl, cg_pass_kernel<DIM, K, double, 8>, gr, bl, 0, s, a, d, mode, last,
                            ini, upd, src, dst)
                 : launch_k(pdl, cg_pass_kernel<DIM, K, double, 32>, gr, bl, 0, s, a, d, mode,
                            last, ini, upd, src, dst);
    else
      e = narrow ? launch_k(pdl, cg_pass_kernel<DIM, K, float, 8>, gr, bl, 0, s, a, d, mode, last,
                            ini, upd, src, dst)
                 : launch_k(pdl, cg_pass_kernel<DIM, K, float, 32>, gr, bl, 0, s, a, d, mode, last,
                            ini, upd, src, dst);
    if (e != cudaSuccess) return e;
    src = dst;
  }
  return cudaGetLastError();
}

template <int DIM, int K>
static cudaError_t cg_init_dk(const lh_ctx* c, const CgArgs& a, cudaStream_t s) {
  if (c->tpc.enabled) return precond_passes<DIM, K>(c, a, true, s);
  cudaError_t e = launch_k(c->use_pdl != 0, cg_reset_kernel, dim3(1), dim3(32), 0, s, c->a.cg,
                           a.gate);
  if (e != cudaSuccess) return e;
  return launch_k(c->use_pdl != 0, cg_jacobi_init_kernel<DIM, K>, dim3(node_grid(c)),
                  dim3(kNodeThreads), 0, s, a);
}

template <int DIM, int K>
static cudaError_t cg_body_dk(const lh_ctx* c, const CgArgs& a, cudaStream_t s) {
  using L = ML<DIM, K>;
  const int eblocks = (int)((c->g.nelem + L::EPB - 1) / L::EPB);
  const bool pdl = c->use_pdl != 0;
  cudaError_t e;
  if (tiles_2d<DIM>(c)) {  // element apply and gather in one kernel over node tiles
    const int64_t blocks = 2 * (int64_t)pass2d_tiles(c->g.nn[0]) * pass2d_tiles(c->g.nn[1]);
    e = launch_k(pdl, cg_apply2d_kernel<K>, dim3((unsigned)blocks), dim3(kLineThreads), 0, s, a);
  } else {
    e = launch_k(pdl, cg_elem_kernel<DIM, K>, dim3(eblocks), dim3(256), 0, s, a);
    if (e == cudaSuccess)
      e = launch_k(pdl, cg_gather_kernel<DIM, K>, dim3(node_grid(c)), dim3(kNodeThreads), 0, s,
                   a);
  }
  if (e != cudaSuccess) return e;
  if (c->tpc.enabled && !c->tpc.exact && fuse_update<DIM>(c))
    return precond_passes<DIM, K>(c, a, false, s, true);
  e = launch_k(pdl, cg_update_kernel<DIM, K>, dim3(node_grid(c)), dim3(kNodeThreads), 0, s, a,
               c->tpc.enabled ? 0 : 1);
  if (e != cudaSuccess) return e;
  if (c->tpc.enabled) {
    if ((e = precond_passes<DIM, K>(c, a, false, s)) != cudaSuccess) return e;
  }
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
  if (c->tpc.B[0] != PB<K>::B) return cudaErrorInvalidValue;
  size_t mx = 0;
  for (int d = 0; d < DIM; ++d) mx = line_smem(c, d) > mx ? line_smem(c, d) : mx;
  return cudaFuncSetAttribute(cg_line_kernel<DIM, K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)mx);
}

// Shared memory of the line passes, set before any stream capture.
cudaError_t cg_prepare(const lh_ctx* c) { LAGH_DISPATCH_CG(cg_prepare_dk, c); }

// One application of the tensor preconditioner on a caller vector: the loop
// passes of the solve (mode 1 reads `in` through CgArgs::r, out through z).
template <int DIM, int K>
static cudaError_t precond_apply_dk(const lh_ctx* c, const double* in, double* out,
                                    cudaStream_t s) {
  CgArgs a = make_args(c, nullptr, nullptr, nullptr);
  a.r = const_cast<double*>(in);
  a.z = out;
  a.standalone = 1;
  return precond_passes<DIM, K>(c, a, false, s);
}

cudaError_t precond_apply(const lh_ctx* c, const double* in, double* out, cudaStream_t s) {
  LAGH_DISPATCH_CG(precond_apply_dk, c, in, out, s);
}

int precond_kernels(const lh_ctx* c) {
  if (!c->tpc.enabled) return 0;
  const int d = c->g.dim;
  return (d == 2 && tiles_2d<2>(c)) ? 1 : d;
}

// The cluster-resident solve: one launch of a cluster of c->cg_cluster CTAs.
template <int DIM, int K>
static cudaError_t cluster_launch_dk(const lh_ctx* c, const CgArgs& a, cudaStream_t s) {
  if constexpr (DIM != 2) {
    return cudaErrorInvalidValue;
  } else {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)c->cg_cluster);
    cfg.blockDim = dim3(kClusterThreads);
    cfg.stream = s;
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)c->cg_cluster;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = c->use_pdl ? 2 : 1;
    return cudaLaunchKernelEx(&cfg, cg_cluster_kernel<DIM, K>, a);
  }
}

static cudaError_t cluster_launch(const lh_ctx* c, const CgArgs& a, cudaStream_t s) {
  LAGH_DISPATCH_CG(cluster_launch_dk, c, a, s);
}

// Cluster size for the cluster-resident solve of this context (0: not used).
template <int DIM, int K>
static int cluster_choose_dk(const lh_ctx* c) {
  if constexpr (DIM != 2) {
    return 0;
  } else {
    auto kern = cg_cluster_kernel<DIM, K>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
        cudaSuccess)
      cudaGetLastError();
    for (int n : {16, 8}) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3((unsigned)n);
      cfg.blockDim = dim3(kClusterThreads);
      cudaLaunchAttribute at;
      at.id = cudaLaunchAttributeClusterDimension;
      at.val.clusterDim.x = (unsigned)n;
      at.val.clusterDim.y = 1;
      at.val.clusterDim.z = 1;
      cfg.attrs = &at;
      cfg.numAttrs = 1;
      int nclusters = 0;
      if (cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg) == cudaSuccess && nclusters > 0)
        return n;
      cudaGetLastError();
    }
    return 0;
  }
}

int cg_cluster_choose(const lh_ctx* c) {
  const int D_ = c->g.dim, K_ = c->g.k;
  if (D_ == 2 && K_ == 1) return cluster_choose_dk<2, 1>(c);
  if (D_ == 2 && K_ == 2) return cluster_choose_dk<2, 2>(c);
  if (D_ == 2 && K_ == 3) return cluster_choose_dk<2, 3>(c);
  return 0;
}

// Eager solve (API): the body is launched in batches and the host polls the
// done flag between batches (or one cluster-resident launch).
cudaError_t cg_solve_eager(const lh_ctx* c, const double* rhs, double* out, cudaStream_t s,
                           int* done_host) {
  CgArgs a = make_args(c, rhs, out, nullptr);
  if (c->cg_cluster > 0) {
    cudaError_t e = cluster_launch(c, a, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(done_host, &c->a.cg->done, sizeof(int),
                                              cudaMemcpyDeviceToHost, s);
    return e == cudaSuccess ? cudaStreamSynchronize(s) : e;
  }
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

// Inside a stream capture on s: the init kernels, the first kUnrolled
// iterations as plain kernels (each returns at once after convergence; the
// last update clears the loop condition if the solve has converged), then a
// WHILE conditional node whose body (captured on `side`) is one CG iteration,
// for solves that need more.  A conditional node relaunches its body graph
// per iteration, so the usual iterations run without it.
constexpr int kUnrolled = 3;

// The iterations a solve usually takes, unrolled ahead of the WHILE node:
// none for Jacobi (tens of iterations), one with the exact inverse, two with
// the FP64 band or the error-free narrow passes (mixed path), three with the
// FP32 band.
static int usual_iterations(const lh_ctx* c) {
  if (!c->tpc.enabled) return 0;
  if (c->tpc.exact) return 1;
  const bool narrow = c->g.dim == 2 ? narrow_passes<2>(c) : narrow_passes<3>(c);
  if (c->tpc.fp64 || (narrow && c->precision == LH_MIXED)) return 2;
  return kUnrolled;
}

cudaError_t cg_solve_capture(const lh_ctx* c, const double* rhs, double* out, const Ctl* gate,
                             cudaStream_t s, cudaStream_t side) {
  CgArgs a = make_args(c, rhs, out, gate);
  if (c->cg_cluster > 0) return cluster_launch(c, a, s);  // one node, no conditional
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
  const int unrolled = usual_iterations(c);
  for (int u = 0; u < unrolled; ++u) {
    CgArgs au = a;
    au.has_cond = (u == unrolled - 1) ? 1 : 0;
    au.cond = h;
    if ((e = cg_body(c, au, s)) != cudaSuccess) return e;
  }
  e = cudaStreamGetCaptureInfo(s, &cs, nullptr, &cap, &deps, nullptr, &ndeps);
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
