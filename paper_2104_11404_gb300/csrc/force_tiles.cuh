// Tile-level device functions of the force and energy kernels (shared by the
// grid kernels of force.cu and the batched stage kernel of batch.cu).
#pragma once

#include <type_traits>

#include "device_util.cuh"
#include "qpoint.cuh"

namespace lagh {


// Layout of a force tile: NTT threads, QPT quadrature points per thread (a
// team of NQD / QPT threads per element), EPB elements.
template <int DIM, int K, bool MIXED, int NTT = 256, int QPT = 1>
struct FL {
  using T = typename std::conditional<MIXED, float, double>::type;
  static constexpr int P = K + 1, NQ = 2 * K;
  static constexpr int ND1 = ipow(P, DIM), ND2 = ipow(K, DIM), NQD = ipow(NQ, DIM);
  static constexpr int TEAM = NQD / QPT;
  static constexpr int EPB = (NTT / TEAM) > 0 ? NTT / TEAM : 1;
  static constexpr int NT = EPB * TEAM;
  static constexpr int PK = P * K;
  // interpolated nodal fields: x, v and (FP64 path) the test vector
  static constexpr int NF = MIXED ? 2 * DIM : 3 * DIM;
  static constexpr int S_INTERP =
      DIM == 2 ? 2 * NF * P * NQ : 2 * NF * P * P * NQ + 3 * NF * P * NQ * NQ;
  static constexpr int S_F1 =
      DIM == 2 ? DIM * DIM * P * NQ : DIM * DIM * P * NQ * NQ + DIM * DIM * P * P * NQ;
  static constexpr int S_FK =
      !MIXED ? 0 : (DIM == 2 ? DIM * DIM * PK * NQ : DIM * DIM * PK * NQ * NQ + DIM * DIM * PK * PK * NQ);
  static constexpr int SCR = S_INTERP > S_F1 ? (S_INTERP > S_FK ? S_INTERP : S_FK)
                                             : (S_F1 > S_FK ? S_F1 : S_FK);
  static constexpr int S_L2 = DIM == 2 ? 2 * K * NQ : 2 * (K * NQ * NQ + K * K * NQ);
  static constexpr size_t al(size_t b) { return (b + 15) & ~size_t(15); }
  // per-element byte sizes
  static constexpr size_t B_XS = al(DIM * ND1 * sizeof(T));
  static constexpr size_t B_VS = B_XS;
  static constexpr size_t B_WS = al(DIM * ND1 * sizeof(double));
  static constexpr size_t B_ES = al(ND2 * sizeof(T));
  static constexpr size_t B_DQ = al(DIM * DIM * NQD * sizeof(T));
  static constexpr size_t B_GQ = al(2 * NQD * sizeof(double));  // FTv and source integrands
  static constexpr size_t B_FK = MIXED ? al(DIM * ND1 * ND2 * sizeof(float)) : 0;
  static constexpr size_t B_SCR = al(SCR * sizeof(T));
  static constexpr size_t B_L2 = al(S_L2 * sizeof(double));
  static constexpr size_t B_ELEM = B_XS + B_VS + B_WS + B_ES + B_DQ + B_GQ + B_FK + B_SCR + B_L2;
  // basis tables; the mixed path adds the products B L and G L of the
  // contractions into F_K: [x][a K + j] = B_a(x) L_j(x) (resp. G_a(x) L_j(x))
  static constexpr size_t B_TAB = al(NQ * P * sizeof(T)) * 2 + al(NQ * K * sizeof(T)) +
                                  al(NQ * K * sizeof(double)) + al(NQ * sizeof(double)) +
                                  al(NQ * sizeof(T)) + (MIXED ? 2 * al(NQ * PK * sizeof(float)) : 0);
  static constexpr size_t BYTES = B_TAB + EPB * B_ELEM + NTT * sizeof(unsigned long long);
};

struct ForceKParams {
  Geom g;
  Phys ph;
  Basis1D b;
  ForceArgs a;
  const double* rho0K;
};

template <typename T>
__device__ __forceinline__ T tab(const double& d, const float& f);
template <>
__device__ __forceinline__ double tab<double>(const double& d, const float&) { return d; }
template <>
__device__ __forceinline__ float tab<float>(const double&, const float& f) { return f; }

// 2D Taylor-Green manufactured source e_src = v.grad(e) of the steady exact
// solution: (pi / (4 (gamma-1))) (cos 3pi x cos pi y - cos pi x cos 3pi y).
__device__ __forceinline__ double tg_source(double X, double Y, double gam) {
  const double pi = 3.141592653589793238462643383279502884;
  return 0.25 * pi / (gam - 1.0) *
         (cos(3.0 * pi * X) * cos(pi * Y) - cos(pi * X) * cos(3.0 * pi * Y));
}

// The same in FP32 for the mixed path, where the source is a right-hand-side
// term evaluated like the stress (four FP64 cosines per point would keep the
// narrow FP64 pipe busy for most of the force kernel).
__device__ __forceinline__ float tg_source_f(float X, float Y, float gam) {
  const float pi = 3.14159265358979f;
  return 0.25f * pi / (gam - 1.0f) *
         (cosf(3.0f * pi * X) * cosf(pi * Y) - cosf(pi * X) * cosf(3.0f * pi * Y));
}

// Synchronisation of one element's team.  A team of at most 32 threads that
// divides 32 lies inside one warp, so a warp barrier orders its shared-memory
// traffic and the warps of the block run their elements independently;
// larger teams use the block barrier.
template <int TEAM>
__device__ __forceinline__ void team_sync() {
  if constexpr (TEAM <= 32 && 32 % TEAM == 0) __syncwarp();
  else __syncthreads();
}

// Minimum of v over the tile into *dst (ordered bits): one atomicMin per warp
// when the block is made of whole warps, else through a shared-memory tree.
template <int NTT>
__device__ __forceinline__ void tile_min_to(unsigned long long v, unsigned long long* sh,
                                            unsigned long long* dst) {
  if constexpr (NTT % 32 == 0) {
    v = warp_min_u64(v);
    if ((threadIdx.x & 31) == 0) atomicMin(dst, v);
  } else {
    block_min_to(v, sh, dst);
  }
}

// Basis tables of the force tiles, written once into the front of the shared
// buffer (the caller synchronises the block before the first tile).
template <int DIM, int K, bool MIXED, int NTT, int QPT = 1>
__device__ __forceinline__ void force_tables(const Basis1D& bas, unsigned char* smem) {
  using F = FL<DIM, K, MIXED, NTT, QPT>;
  using T = typename F::T;
  constexpr int P = F::P, NQ = F::NQ;
  unsigned char* sp = smem;
  T* Bs = reinterpret_cast<T*>(sp); sp += F::al(NQ * P * sizeof(T));
  T* Gs = reinterpret_cast<T*>(sp); sp += F::al(NQ * P * sizeof(T));
  T* Ls = reinterpret_cast<T*>(sp); sp += F::al(NQ * K * sizeof(T));
  double* Ld = reinterpret_cast<double*>(sp); sp += F::al(NQ * K * sizeof(double));
  double* Wd = reinterpret_cast<double*>(sp); sp += F::al(NQ * sizeof(double));
  T* Wt = reinterpret_cast<T*>(sp);
  const int tid = threadIdx.x;
  for (int i = tid; i < NQ * P; i += blockDim.x) {
    int q = i / P, a = i - q * P;
    Bs[i] = tab<T>(bas.B[q][a], bas.Bf[q][a]);
    Gs[i] = tab<T>(bas.G[q][a], bas.Gf[q][a]);
  }
  for (int i = tid; i < NQ * K; i += blockDim.x) {
    int q = i / K, j = i - q * K;
    Ls[i] = tab<T>(bas.L[q][j], bas.Lf[q][j]);
    Ld[i] = bas.L[q][j];
  }
  for (int i = tid; i < NQ; i += blockDim.x) {
    Wd[i] = bas.W[i];
    Wt[i] = tab<T>(bas.W[i], bas.Wf[i]);
  }
  if constexpr (MIXED) {
    constexpr int PK = F::PK;
    sp += F::al(NQ * sizeof(T));
    float* BLt = reinterpret_cast<float*>(sp); sp += F::al(NQ * PK * sizeof(float));
    float* GLt = reinterpret_cast<float*>(sp);
    for (int i = tid; i < NQ * PK; i += blockDim.x) {
      const int x = i / PK, u = i - x * PK, a = u / K, j = u - a * K;
      BLt[i] = __fmul_rn(bas.Bf[x][a], bas.Lf[x][j]);
      GLt[i] = __fmul_rn(bas.Gf[x][a], bas.Lf[x][j]);
    }
  }
}

// One tile of EPB element slots [slot0, slot0 + EPB) of the force evaluation,
// by all NTT threads of the block (the grid kernel below uses one tile per
// block; the batched stage kernel loops over the tiles of an instance).
// SRC32: the mixed path evaluates the Taylor-Green energy source in FP32
// (the grid kernel); otherwise it is evaluated in FP64 (the batched kernel,
// whose point-blast instances carry no source, keeps its code unchanged).
template <int DIM, int K, bool MIXED, int NTT, int QPT = 1, bool SRC32 = false>
__device__ __forceinline__ void force_tile(const Geom& g, const Phys& ph, const Basis1D& bas,
                                           const ForceArgs& A, const double* rho0Kp,
                                           unsigned char* smem, int64_t slot0) {
  using F = FL<DIM, K, MIXED, NTT, QPT>;
  using T = typename F::T;
  constexpr int P = F::P, NQ = F::NQ, ND1 = F::ND1, ND2 = F::ND2, NQD = F::NQD;
  constexpr int TEAM = F::TEAM;
  constexpr int NF = F::NF;
  struct Prm { const Phys& ph; const Basis1D& b; const double* rho0K; } prm{ph, bas, rho0Kp};
  unsigned char* sp = smem;
  T* Bs = reinterpret_cast<T*>(sp); sp += F::al(NQ * P * sizeof(T));
  T* Gs = reinterpret_cast<T*>(sp); sp += F::al(NQ * P * sizeof(T));
  T* Ls = reinterpret_cast<T*>(sp); sp += F::al(NQ * K * sizeof(T));
  double* Ld = reinterpret_cast<double*>(sp); sp += F::al(NQ * K * sizeof(double));
  double* Wd = reinterpret_cast<double*>(sp); sp += F::al(NQ * sizeof(double));
  T* Wt = reinterpret_cast<T*>(sp); sp += F::al(NQ * sizeof(T));
  const float* BLt = nullptr;
  const float* GLt = nullptr;
  if constexpr (MIXED) {
    BLt = reinterpret_cast<const float*>(sp); sp += F::al(NQ * F::PK * sizeof(float));
    GLt = reinterpret_cast<const float*>(sp); sp += F::al(NQ * F::PK * sizeof(float));
  }
  unsigned long long* red = reinterpret_cast<unsigned long long*>(smem + F::B_TAB + F::EPB * F::B_ELEM);

  const int tid = threadIdx.x;
  const int le = tid / TEAM;       // element of this thread's team
  const int tq = tid - le * TEAM;  // team rank: quadrature points tq, tq + TEAM, ...
  unsigned char* ep = sp + le * F::B_ELEM;
  T* xs = reinterpret_cast<T*>(ep); ep += F::B_XS;
  T* vs = reinterpret_cast<T*>(ep); ep += F::B_VS;
  double* ws = reinterpret_cast<double*>(ep); ep += F::B_WS;
  T* es = reinterpret_cast<T*>(ep); ep += F::B_ES;
  T* dq = reinterpret_cast<T*>(ep); ep += F::B_DQ;
  double* gq = reinterpret_cast<double*>(ep); ep += F::B_GQ;  // [2][NQD]
  float* fk = reinterpret_cast<float*>(ep); ep += F::B_FK;
  T* scr = reinterpret_cast<T*>(ep); ep += F::B_SCR;
  double* l2s = reinterpret_cast<double*>(ep);

  const int64_t slot = slot0 + le;
  const bool active = le < F::EPB && slot < A.nslots;
  const int64_t el = active ? (A.list ? (int64_t)A.list[slot] : slot) : 0;
  int E[3] = {0, 0, 0};
  elem_ijk(g, el, E);
  const bool with_w = A.vtest != nullptr;

  // ---- stage element data ----
  double x0[DIM];  // element origin (mixed path subtracts it before rounding)
  {
    int64_t n0 = elem_node<K>(g, E, 0, 0, 0);
    for (int c = 0; c < DIM; ++c) x0[c] = MIXED ? A.x[c * g.nnodes + n0] : 0.0;
  }
  if (active) {
    // every load issued before the shared-memory stores (a load per loop
    // iteration behind the previous iteration's stores runs one at a time)
    constexpr int PS = (DIM * ND1 + TEAM - 1) / TEAM, PE = (ND2 + TEAM - 1) / TEAM;
    double xv[PS], vv[PS], wv[PS], ev[PE];
#pragma unroll
    for (int j = 0; j < PS; ++j) {
      const int w = tq + j * TEAM;
      xv[j] = vv[j] = wv[j] = 0.0;
      if (w < DIM * ND1) {
        const int c = w / ND1, i = w - c * ND1;
        const int a = i % P, b = (i / P) % P, cc = DIM == 3 ? i / (P * P) : 0;
        const int64_t k = c * g.nnodes + elem_node<K>(g, E, a, b, cc);
        xv[j] = A.x[k];
        vv[j] = A.v[k];
        if (with_w) wv[j] = A.vtest[k];
      }
    }
#pragma unroll
    for (int j = 0; j < PE; ++j) ev[j] = tq + j * TEAM < ND2 ? A.e[el * ND2 + tq + j * TEAM] : 0.0;
#pragma unroll
    for (int j = 0; j < PS; ++j) {
      const int w = tq + j * TEAM;
      if (w < DIM * ND1) {
        xs[w] = from_double<T>(xv[j] - x0[w / ND1]);
        vs[w] = from_double<T>(vv[j]);
        if (with_w) ws[w] = wv[j];
      }
    }
#pragma unroll
    for (int j = 0; j < PE; ++j)
      if (tq + j * TEAM < ND2) es[tq + j * TEAM] = from_double<T>(ev[j]);
  }
  team_sync<TEAM>();

  // ---- reference gradients at the quadrature points (sum factorisation) ----
  // fields f: [0, DIM) x, [DIM, 2 DIM) v, [2 DIM, 3 DIM) test vector (FP64 path)
  auto field = [&](int f, int i) -> T {
    if (f < DIM) return xs[f * ND1 + i];
    if (f < 2 * DIM) return vs[(f - DIM) * ND1 + i];
    return (T)ws[(f - 2 * DIM) * ND1 + i];
  };
  const int nf = (MIXED || !with_w) ? 2 * DIM : 3 * DIM;
  if constexpr (DIM == 2) {
    T* TB = scr;
    T* TG = scr + NF * P * NQ;
    if (active)
      for (int w = tq; w < nf * P * NQ; w += TEAM) {
        int x_ = w % NQ, b = (w / NQ) % P, f = w / (NQ * P);
        T sb = T(0), sg = T(0);
        for (int a = 0; a < P; ++a) {
          T u = field(f, b * P + a);
          sb += Bs[x_ * P + a] * u;
          sg += Gs[x_ * P + a] * u;
        }
        TB[(f * P + b) * NQ + x_] = sb;
        TG[(f * P + b) * NQ + x_] = sg;
      }
  } else {
    T* TB = scr;
    T* TG = TB + NF * P * P * NQ;
    T* PBB = TG + NF * P * P * NQ;
    T* PGB = PBB + NF * P * NQ * NQ;
    T* PBG = PGB + NF * P * NQ * NQ;
    if (active)
      for (int w = tq; w < nf * P * P * NQ; w += TEAM) {
        int x_ = w % NQ, r = w / NQ;  // r = (f * P + cz) * P + b
        int b = r % P, fz = r / P;    // fz = f * P + cz
        T sb = T(0), sg = T(0);
        int f = fz / P, cz = fz - f * P;
        for (int a = 0; a < P; ++a) {
          T u = field(f, (cz * P + b) * P + a);
          sb += Bs[x_ * P + a] * u;
          sg += Gs[x_ * P + a] * u;
        }
        TB[r * NQ + x_] = sb;
        TG[r * NQ + x_] = sg;
      }
    team_sync<TEAM>();
    if (active)
      for (int w = tq; w < nf * P * NQ * NQ; w += TEAM) {
        int x_ = w % NQ, y_ = (w / NQ) % NQ, fz = w / (NQ * NQ);
        T bb = T(0), gb = T(0), bg = T(0);
        for (int b = 0; b < P; ++b) {
          T tb = TB[(fz * P + b) * NQ + x_], tg = TG[(fz * P + b) * NQ + x_];
          bb += Bs[y_ * P + b] * tb;
          gb += Bs[y_ * P + b] * tg;
          bg += Gs[y_ * P + b] * tb;
        }
        PBB[w] = bb;
        PGB[w] = gb;
        PBG[w] = bg;
      }
  }
  team_sync<TEAM>();

  // ---- quadrature-point physics, for each of the thread's QPT points ----
  double tau_q = t_inf<double>();
  int flags = 0;
  if (active)
#pragma unroll
    for (int qq = 0; qq < QPT; ++qq) {
      const int q = tq + qq * TEAM;  // quadrature point
      const int qx = q % NQ, qy = (q / NQ) % NQ, qz = DIM == 3 ? q / (NQ * NQ) : 0;
      T grad[NF][DIM];
      T xval[DIM];
      if constexpr (DIM == 2) {
        const T* TB = scr;
        const T* TG = scr + NF * P * NQ;
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          if (f >= nf) break;
          T d0 = T(0), d1 = T(0), vv = T(0);
          for (int b = 0; b < P; ++b) {
            T tb = TB[(f * P + b) * NQ + qx], tg = TG[(f * P + b) * NQ + qx];
            d0 += Bs[qy * P + b] * tg;
            d1 += Gs[qy * P + b] * tb;
            vv += Bs[qy * P + b] * tb;
          }
          grad[f][0] = d0;
          grad[f][1] = d1;
          if (f < DIM) xval[f] = vv;
        }
      } else {
        const T* PBB = scr + 2 * NF * P * P * NQ;
        const T* PGB = PBB + NF * P * NQ * NQ;
        const T* PBG = PGB + NF * P * NQ * NQ;
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          if (f >= nf) break;
          T d0 = T(0), d1 = T(0), d2 = T(0), vv = T(0);
          for (int cz = 0; cz < P; ++cz) {
            int idx = ((f * P + cz) * NQ + qy) * NQ + qx;
            d0 += Bs[qz * P + cz] * PGB[idx];
            d1 += Bs[qz * P + cz] * PBG[idx];
            d2 += Gs[qz * P + cz] * PBB[idx];
            vv += Bs[qz * P + cz] * PBB[idx];
          }
          grad[f][0] = d0;
          grad[f][1] = d1;
          grad[f][2] = d2;
          if (f < DIM) xval[f] = vv;
        }
      }
      T e_q = T(0);
      for (int j = 0; j < ND2; ++j) {
        int jx = j % K, jy = (j / K) % K, jz = DIM == 3 ? j / (K * K) : 0;
        T phi = Ls[qx * K + jx] * Ls[qy * K + jy];
        if (DIM == 3) phi *= Ls[qz * K + jz];
        e_q += es[j] * phi;
      }
      T J[DIM][DIM], Gv[DIM][DIM], J0i[DIM], sigma[DIM][DIM], tau;
      for (int c = 0; c < DIM; ++c) {
        J0i[c] = tab<T>(g.J0inv[c], g.J0invf[c]);
        for (int m = 0; m < DIM; ++m) {
          J[c][m] = grad[c][m];
          Gv[c][m] = grad[DIM + c][m];
        }
      }
      const T rho0K = from_double<T>(prm.rho0K[el]);
      if (A.mode == kForceFull) {
        const T pref = (MIXED && A.p_ref != nullptr) ? from_double<T>(*A.p_ref) : T(0);
        const T gam = A.gammaE != nullptr ? from_double<T>(A.gammaE[el])
                                          : pconst<T>(prm.ph.gamma, prm.ph.gammaf);
        flags |= qpoint_physics<T, DIM>(J, Gv, e_q, rho0K, gam, prm.ph, J0i,
                                        tab<T>(g.ell0, g.ell0f), T(1) / T(K), pref, sigma, tau);
        const double tq_d = to_double(tau);
        tau_q = tq_d < tau_q ? tq_d : tau_q;
      } else {
        // reference pressure only: sigma = -p_ref I
        const T pref = from_double<T>(*A.p_ref);
        for (int c = 0; c < DIM; ++c)
          for (int n = 0; n < DIM; ++n) sigma[c][n] = (c == n) ? -pref : T(0);
      }
      const T alphaT = DIM == 3 ? Wt[qx] * Wt[qy] * Wt[qz] : Wt[qx] * Wt[qy];
      T Aj[DIM][DIM];
      adj_of<T, DIM>(J, Aj);
      for (int c = 0; c < DIM; ++c)
        for (int m = 0; m < DIM; ++m) {
          T acc = T(0);
          for (int n = 0; n < DIM; ++n) acc += sigma[c][n] * Aj[m][n];
          dq[(c * DIM + m) * NQD + q] = alphaT * acc;
        }
      if (!MIXED && A.D != nullptr)
        for (int cm = 0; cm < DIM * DIM; ++cm)
          A.D[(el * DIM * DIM + cm) * NQD + q] = (double)dq[cm * NQD + q];
      if (!MIXED && with_w) {
        double gsum = 0.0;
        for (int c = 0; c < DIM; ++c)
          for (int m = 0; m < DIM; ++m)
            gsum += (double)dq[(c * DIM + m) * NQD + q] * (double)grad[2 * DIM + c][m];
        gq[q] = gsum;
      }
      if (A.srcE != nullptr && DIM == 2) {
        if constexpr (MIXED && SRC32) {
          const float X = __fadd_rn(from_double<float>(x0[0]), xval[0]);
          const float Y = __fadd_rn(from_double<float>(x0[1]), xval[1]);
          gq[NQD + q] = to_double(alphaT * rho0K * tg_source_f(X, Y, prm.ph.gammaf));
        } else {
          const double alpha = Wd[qx] * Wd[qy];
          double X = x0[0] + to_double(xval[0]), Y = x0[1] + to_double(xval[1]);
          gq[NQD + q] = alpha * prm.rho0K[el] * tg_source(X, Y, prm.ph.gamma);
        }
      }
    }
  // time-step estimate and error flags of the block
  if (A.tau_bits != nullptr) tile_min_to<NTT>(tau_to_bits(tau_q), red, A.tau_bits);
  if (flags && A.status != nullptr) atomicOr(A.status, flags);
  team_sync<TEAM>();

  // ---- transposed contractions ----
  if constexpr (!MIXED) {
    if (A.F1E == nullptr) goto l2_part;
    {
    // F.1 rows: F1[c][i] = sum_q sum_m D[c][m](q) d_m w_i(q)
    if constexpr (DIM == 2) {
      T* Y = scr;
      if (active)
        for (int w = tq; w < DIM * DIM * P * NQ; w += TEAM) {
          int x_ = w % NQ, b = (w / NQ) % P, cm = w / (NQ * P), m = cm % DIM;
          const T* X = (m == 1) ? Gs : Bs;
          T s = T(0);
          for (int y_ = 0; y_ < NQ; ++y_) s += X[y_ * P + b] * dq[cm * NQD + y_ * NQ + x_];
          Y[w] = s;
        }
      team_sync<TEAM>();
      if (active)
        for (int w = tq; w < DIM * ND1; w += TEAM) {
          int c = w / ND1, i = w - c * ND1, a = i % P, b = i / P;
          T s = T(0);
          for (int m = 0; m < DIM; ++m) {
            const T* X = (m == 0) ? Gs : Bs;
            for (int x_ = 0; x_ < NQ; ++x_) s += X[x_ * P + a] * Y[(((c * DIM + m) * P + b) * NQ) + x_];
          }
          double* o = &A.F1E[(slot * DIM + c) * ND1 + i];
          *o = A.accumulate ? *o + (double)s : (double)s;
        }
    } else {
      T* Y = scr;
      T* Z = scr + DIM * DIM * P * NQ * NQ;
      if (active)
        for (int w = tq; w < DIM * DIM * P * NQ * NQ; w += TEAM) {
          int x_ = w % NQ, y_ = (w / NQ) % NQ, cz = (w / (NQ * NQ)) % P, cm = w / (NQ * NQ * P);
          int m = cm % DIM;
          const T* X = (m == 2) ? Gs : Bs;
          T s = T(0);
          for (int z_ = 0; z_ < NQ; ++z_)
            s += X[z_ * P + cz] * dq[cm * NQD + (z_ * NQ + y_) * NQ + x_];
          Y[w] = s;
        }
      team_sync<TEAM>();
      if (active)
        for (int w = tq; w < DIM * DIM * P * P * NQ; w += TEAM) {
          int x_ = w % NQ, b = (w / NQ) % P, cz = (w / (NQ * P)) % P, cm = w / (NQ * P * P);
          int m = cm % DIM;
          const T* X = (m == 1) ? Gs : Bs;
          T s = T(0);
          for (int y_ = 0; y_ < NQ; ++y_)
            s += X[y_ * P + b] * Y[((cm * P + cz) * NQ + y_) * NQ + x_];
          Z[w] = s;
        }
      team_sync<TEAM>();
      if (active)
        for (int w = tq; w < DIM * ND1; w += TEAM) {
          int c = w / ND1, i = w - c * ND1, a = i % P, b = (i / P) % P, cz = i / (P * P);
          T s = T(0);
          for (int m = 0; m < DIM; ++m) {
            const T* X = (m == 0) ? Gs : Bs;
            for (int x_ = 0; x_ < NQ; ++x_)
              s += X[x_ * P + a] * Z[((((c * DIM + m) * P + cz) * P + b) * NQ) + x_];
          }
          double* o = &A.F1E[(slot * DIM + c) * ND1 + i];
          *o = A.accumulate ? *o + (double)s : (double)s;
        }
    }
    }
  } else {
    // Mixed: F_K[(c,i), j] = sum_q phi_j(q) sum_m D[c][m](q) d_m w_i(q) in FP32,
    // one direction at a time (sum factorisation).  The factor of direction
    // d is B_a L_j, or G_a L_j along the derivative's direction m = d, taken
    // from the product tables (each product rounded once, as a product
    // formed on the fly).  A work item holds the NQ points of one line in
    // registers and produces all PK = P K (a, j) outputs of that line; the
    // terms of every sum are added in point order (m, then the point, in the
    // last direction).
    constexpr int PK = F::PK;
    if constexpr (DIM == 2) {
      T* Y = scr;  // [cm][u = (b, jy)][x]
      if (active)
        for (int it = tq; it < DIM * DIM * NQ; it += TEAM) {
          const int x_ = it % NQ, cm = it / NQ, m = cm % DIM;
          const float* Ty = (m == 1) ? GLt : BLt;
          float dv[NQ];
#pragma unroll
          for (int y_ = 0; y_ < NQ; ++y_) dv[y_] = dq[cm * NQD + y_ * NQ + x_];
#pragma unroll
          for (int u = 0; u < PK; ++u) {
            float acc = 0.0f;
#pragma unroll
            for (int y_ = 0; y_ < NQ; ++y_) acc = fmaf(Ty[y_ * PK + u], dv[y_], acc);
            Y[(cm * PK + u) * NQ + x_] = acc;
          }
        }
      team_sync<TEAM>();
      if (active)
        for (int it = tq; it < DIM * PK; it += TEAM) {
          const int c = it / PK, u = it - c * PK, b = u / K, jy = u - b * K;
          float yv[DIM][NQ];
#pragma unroll
          for (int m = 0; m < DIM; ++m)
#pragma unroll
            for (int x_ = 0; x_ < NQ; ++x_) yv[m][x_] = Y[((c * DIM + m) * PK + u) * NQ + x_];
#pragma unroll
          for (int v = 0; v < PK; ++v) {
            const int a = v / K, jx = v - a * K;
            float acc = 0.0f;
#pragma unroll
            for (int m = 0; m < DIM; ++m) {
              const float* Tx = (m == 0) ? GLt : BLt;
#pragma unroll
              for (int x_ = 0; x_ < NQ; ++x_) acc = fmaf(Tx[x_ * PK + v], yv[m][x_], acc);
            }
            fk[(c * ND1 + a + P * b) * ND2 + jx + K * jy] = acc;
          }
        }
    } else {
      T* Y = scr;                                 // [cm][uz][y][x]
      T* Z = scr + DIM * DIM * PK * NQ * NQ;      // [cm][uz][uy][x]
      if (active)
        for (int it = tq; it < DIM * DIM * NQ * NQ; it += TEAM) {
          const int x_ = it % NQ, y_ = (it / NQ) % NQ, cm = it / (NQ * NQ), m = cm % DIM;
          const float* Tz = (m == 2) ? GLt : BLt;
          float dv[NQ];
#pragma unroll
          for (int z_ = 0; z_ < NQ; ++z_) dv[z_] = dq[cm * NQD + (z_ * NQ + y_) * NQ + x_];
#pragma unroll
          for (int u = 0; u < PK; ++u) {
            float acc = 0.0f;
#pragma unroll
            for (int z_ = 0; z_ < NQ; ++z_) acc = fmaf(Tz[z_ * PK + u], dv[z_], acc);
            Y[((cm * PK + u) * NQ + y_) * NQ + x_] = acc;
          }
        }
      team_sync<TEAM>();
      if (active)
        for (int it = tq; it < DIM * DIM * PK * NQ; it += TEAM) {
          const int x_ = it % NQ, uz = (it / NQ) % PK, cm = it / (NQ * PK), m = cm % DIM;
          const float* Ty = (m == 1) ? GLt : BLt;
          float yv[NQ];
#pragma unroll
          for (int y_ = 0; y_ < NQ; ++y_) yv[y_] = Y[((cm * PK + uz) * NQ + y_) * NQ + x_];
#pragma unroll
          for (int uy = 0; uy < PK; ++uy) {
            float acc = 0.0f;
#pragma unroll
            for (int y_ = 0; y_ < NQ; ++y_) acc = fmaf(Ty[y_ * PK + uy], yv[y_], acc);
            Z[((cm * PK + uz) * PK + uy) * NQ + x_] = acc;
          }
        }
      team_sync<TEAM>();
      if (active)
        for (int it = tq; it < DIM * PK * PK; it += TEAM) {
          const int uy = it % PK, uz = (it / PK) % PK, c = it / (PK * PK);
          const int b = uy / K, jy = uy - b * K, cz = uz / K, jz = uz - cz * K;
          float zv[DIM][NQ];
#pragma unroll
          for (int m = 0; m < DIM; ++m)
#pragma unroll
            for (int x_ = 0; x_ < NQ; ++x_)
              zv[m][x_] = Z[((((c * DIM + m) * PK + uz) * PK + uy) * NQ) + x_];
#pragma unroll
          for (int v = 0; v < PK; ++v) {
            const int a = v / K, jx = v - a * K;
            float acc = 0.0f;
#pragma unroll
            for (int m = 0; m < DIM; ++m) {
              const float* Tx = (m == 0) ? GLt : BLt;
#pragma unroll
              for (int x_ = 0; x_ < NQ; ++x_) acc = fmaf(Tx[x_ * PK + v], zv[m][x_], acc);
            }
            fk[(c * ND1 + a + P * (b + P * cz)) * ND2 + jx + K * (jy + K * jz)] = acc;
          }
        }
    }
    team_sync<TEAM>();
    if (active) {
      if (A.FK != nullptr)
        for (int w = tq; w < DIM * ND1 * ND2; w += TEAM) A.FK[el * (DIM * ND1 * ND2) + w] = fk[w];
      // F.1 = row sums: error-free FP32 sums (the rounding errors collected
      // apart), widened to FP64 (the FP32 entries summed to ~2^-48)
      for (int w = tq; w < DIM * ND1; w += TEAM) {
        float S = fk[w * ND2], C = 0.0f;
        for (int j = 1; j < ND2; ++j) {
          float s2, e2;
          two_sum_f(S, fk[w * ND2 + j], s2, e2);
          S = s2;
          C = __fadd_rn(C, e2);
        }
        A.F1E[slot * DIM * ND1 + w] = f2d_exact(S) + f2d_exact(C);
      }
      // F^T w in FP64
      if (with_w)
        for (int j = tq; j < ND2; j += TEAM) {
          double s = 0.0;
          for (int ci = 0; ci < DIM * ND1; ++ci) s = fma(f2d_exact(fk[ci * ND2 + j]), ws[ci], s);
          A.FTvE[slot * ND2 + j] = s;
        }
    }
  }

  // ---- L2 contractions (FP64): F^T w (FP64 path) and the energy source ----
l2_part:
  const bool do_ftv = (!MIXED) && with_w;
  const bool do_src = (A.srcE != nullptr) && DIM == 2;
  if (do_ftv || do_src) {
    team_sync<TEAM>();
    // field 0: F^T w integrand, field 1: source integrand
    if constexpr (DIM == 2) {
      double* R1 = l2s;  // [2][K][NQ]
      if (active)
        for (int w = tq; w < 2 * K * NQ; w += TEAM) {
          int y_ = w % NQ, jx = (w / NQ) % K, fld = w / (NQ * K);
          double s = 0.0;
          for (int x_ = 0; x_ < NQ; ++x_) s += Ld[x_ * K + jx] * gq[fld * NQD + y_ * NQ + x_];
          R1[w] = s;
        }
      team_sync<TEAM>();
      if (active)
        for (int w = tq; w < 2 * ND2; w += TEAM) {
          int fld = w / ND2, j = w - fld * ND2, jx = j % K, jy = j / K;
          if ((fld == 0 && !do_ftv) || (fld == 1 && !do_src)) continue;
          double s = 0.0;
          for (int y_ = 0; y_ < NQ; ++y_) s += Ld[y_ * K + jy] * R1[(fld * K + jx) * NQ + y_];
          if (fld == 0) A.FTvE[slot * ND2 + j] = A.accumulate ? A.FTvE[slot * ND2 + j] + s : s;
          else A.srcE[el * ND2 + j] = s;
        }
    } else {
      double* R1 = l2s;                 // [2][K][NQ][NQ]
      double* R2 = l2s + 2 * K * NQ * NQ;  // [2][K][K][NQ]
      if (active)
        for (int w = tq; w < 2 * K * NQ * NQ; w += TEAM) {
          int y_ = w % NQ, z_ = (w / NQ) % NQ, jx = (w / (NQ * NQ)) % K, fld = w / (NQ * NQ * K);
          double s = 0.0;
          for (int x_ = 0; x_ < NQ; ++x_)
            s += Ld[x_ * K + jx] * gq[fld * NQD + (z_ * NQ + y_) * NQ + x_];
          R1[w] = s;
        }
      team_sync<TEAM>();
      if (active)
        for (int w = tq; w < 2 * K * K * NQ; w += TEAM) {
          int z_ = w % NQ, jx = (w / NQ) % K, jy = (w / (NQ * K)) % K, fld = w / (NQ * K * K);
          double s = 0.0;
          for (int y_ = 0; y_ < NQ; ++y_)
            s += Ld[y_ * K + jy] * R1[((fld * K + jx) * NQ + z_) * NQ + y_];
          R2[w] = s;
        }
      team_sync<TEAM>();
      if (active)
        for (int w = tq; w < 2 * ND2; w += TEAM) {
          int fld = w / ND2, j = w - fld * ND2, jx = j % K, jy = (j / K) % K, jz = j / (K * K);
          if ((fld == 0 && !do_ftv) || (fld == 1 && !do_src)) continue;
          double s = 0.0;
          for (int z_ = 0; z_ < NQ; ++z_)
            s += Ld[z_ * K + jz] * R2[((fld * K + jy) * K + jx) * NQ + z_];
          if (fld == 0) A.FTvE[slot * ND2 + j] = A.accumulate ? A.FTvE[slot * ND2 + j] + s : s;
          else A.srcE[el * ND2 + j] = s;
        }
    }
  }
  team_sync<TEAM>();  // the team reuses its element area in the next tile
}

template <int DIM, int K, bool MIXED, int NTT = 256>
__global__ void __launch_bounds__(FL<DIM, K, MIXED, NTT>::NT)
force_kernel(const ForceKParams prm) {
  pdl_enter();
  using F = FL<DIM, K, MIXED, NTT>;
  if (prm.a.ctl != nullptr && prm.a.ctl->done) return;
  extern __shared__ __align__(16) unsigned char smem[];
  force_tables<DIM, K, MIXED, F::NT>(prm.b, smem);
  __syncthreads();
  force_tile<DIM, K, MIXED, F::NT, 1, true>(prm.g, prm.ph, prm.b, prm.a, prm.rho0K, smem,
                                            (int64_t)blockIdx.x * F::EPB);
}

// ------------------------------------------------------------- gather ----

template <int DIM, int K>
__global__ void gather_kernel(Geom g, const double* __restrict__ E, double* __restrict__ out,
                              double scale, int apply_bc, const Ctl* ctl) {
  pdl_enter();
  if (ctl != nullptr && ctl->done) return;
  int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (node >= g.nnodes) return;
  int I[3];
  node_ijk(g, node, I);
  for (int c = 0; c < DIM; ++c) {
    double val = (apply_bc && essential(g, I, c)) ? 0.0 : scale * gather_node<DIM, K>(g, E, I, c);
    out[c * g.nnodes + node] = val;
  }
}

// ------------------------------------------------------- energy update ----

// e_out = e_base + coef * M_E^{-1} (F^T w + src) per element.  One team of
// NQ^DIM threads per element (same mapping as the force kernel) forms F^T w;
// the FP64 combination and M_E^{-1} then run over the tile's (element, row)
// pairs with every lane busy (an FP64 instruction costs its warp the same
// pipe time however few of its lanes are active).
template <int DIM, int K, bool MIXED, int NTT = 256>
struct EL {
  static constexpr int P = K + 1, NQ = 2 * K;
  static constexpr int ND1 = ipow(P, DIM), ND2 = ipow(K, DIM), NQD = ipow(NQ, DIM);
  static constexpr int EPB = (NTT / NQD) > 0 ? NTT / NQD : 1;
  static constexpr int NT = EPB * NQD;
  // interpolated fields: w (FP64 path); w and x (mixed path, reference pressure)
  static constexpr int NFI = MIXED ? 2 * DIM : DIM;
  static constexpr int S_INTERP = DIM == 2 ? 2 * NFI * P * NQ
                                           : 2 * NFI * P * P * NQ + 3 * NFI * P * NQ * NQ;
  static constexpr int S_L2 = DIM == 2 ? K * NQ : K * NQ * NQ + K * K * NQ;
  static constexpr size_t al(size_t b) { return (b + 15) & ~size_t(15); }
  // per element: staged fields, interpolation scratch, point integrands,
  // L2 scratch, F^T w, the mixed path's chunk sums and reference-pressure part
  static constexpr size_t B_ELEM = al(NFI * ND1 * 8) + al(S_INTERP * 8) + al(NQD * 8) +
                                   al(S_L2 * 8) + al(ND2 * 8) +
                                   (MIXED ? al(NQD * 8) + al(ND2 * 8) : 0);
  static constexpr size_t B_TAB = 3 * al(NQ * P * 8) + al(NQ * K * 8) + al(81 * 8);
  static constexpr size_t BYTES = B_TAB + EPB * B_ELEM;
};

struct EnergyKParams {
  Geom g;
  Basis1D b;
  EnergyArgs a;
  const double* rho0K;
};

// Basis tables of the energy tiles (written once; the caller synchronises).
template <int DIM, int K, bool MIXED, int NTT>
__device__ __forceinline__ void energy_tables(const Basis1D& bas, unsigned char* smem) {
  using F = EL<DIM, K, MIXED, NTT>;
  constexpr int P = F::P, NQ = F::NQ, ND2 = F::ND2;
  unsigned char* sp = smem;
  double* Bs = reinterpret_cast<double*>(sp); sp += F::al(NQ * P * 8);
  double* Gs = reinterpret_cast<double*>(sp); sp += F::al(NQ * P * 8);
  double* Wd = reinterpret_cast<double*>(sp); sp += F::al(NQ * P * 8);
  double* Ls = reinterpret_cast<double*>(sp); sp += F::al(NQ * K * 8);
  double* Mi = reinterpret_cast<double*>(sp);
  const int tid = threadIdx.x;
  for (int i = tid; i < NQ * P; i += blockDim.x) {
    Bs[i] = bas.B[i / P][i % P];
    Gs[i] = bas.G[i / P][i % P];
  }
  for (int i = tid; i < NQ; i += blockDim.x) Wd[i] = bas.W[i];
  for (int i = tid; i < NQ * K; i += blockDim.x) Ls[i] = bas.L[i / K][i % K];
  for (int i = tid; i < ND2 * ND2; i += blockDim.x) Mi[i] = bas.MEinv[i];
}

// Reference gradients of nf FP64 fields (fields[f][ND1], staged by the team)
// at the team's quadrature point: grad[f][m] = d_m u_f (sum factorisation in
// the team's scratch).  Every thread of the block calls it.
template <int DIM, int K, int NQD, int NFMAX>
__device__ __forceinline__ void interp_grads(const double* fields, int nf, double* scr,
                                             const double* Bs, const double* Gs, int tq,
                                             bool active, double (&grad)[NFMAX][DIM]) {
  constexpr int P = K + 1, NQ = 2 * K, ND1 = ipow(P, DIM);
  const int qx = tq % NQ, qy = (tq / NQ) % NQ, qz = DIM == 3 ? tq / (NQ * NQ) : 0;
  if constexpr (DIM == 2) {
    double* TB = scr;
    double* TG = scr + nf * P * NQ;
    if (active)
      for (int w = tq; w < nf * P * NQ; w += NQD) {
        int x_ = w % NQ, b = (w / NQ) % P, f = w / (NQ * P);
        double sb = 0.0, sg = 0.0;
        for (int a = 0; a < P; ++a) {
          double u = fields[f * ND1 + b * P + a];
          sb += Bs[x_ * P + a] * u;
          sg += Gs[x_ * P + a] * u;
        }
        TB[w] = sb;
        TG[w] = sg;
      }
    team_sync<NQD>();
    if (active)
      for (int f = 0; f < nf; ++f) {
        double d0 = 0.0, d1 = 0.0;
        for (int b = 0; b < P; ++b) {
          d0 += Bs[qy * P + b] * TG[(f * P + b) * NQ + qx];
          d1 += Gs[qy * P + b] * TB[(f * P + b) * NQ + qx];
        }
        grad[f][0] = d0;
        grad[f][1] = d1;
      }
  } else {
    double* TB = scr;
    double* TG = TB + nf * P * P * NQ;
    double* PBB = TG + nf * P * P * NQ;
    double* PGB = PBB + nf * P * NQ * NQ;
    double* PBG = PGB + nf * P * NQ * NQ;
    if (active)
      for (int w = tq; w < nf * P * P * NQ; w += NQD) {
        int x_ = w % NQ, r = w / NQ, b = r % P, fz = r / P;
        int f = fz / P, cz = fz - f * P;
        double sb = 0.0, sg = 0.0;
        for (int a = 0; a < P; ++a) {
          double u = fields[f * ND1 + (cz * P + b) * P + a];
          sb += Bs[x_ * P + a] * u;
          sg += Gs[x_ * P + a] * u;
        }
        TB[w] = sb;
        TG[w] = sg;
      }
    team_sync<NQD>();
    if (active)
      for (int w = tq; w < nf * P * NQ * NQ; w += NQD) {
        int x_ = w % NQ, y_ = (w / NQ) % NQ, fz = w / (NQ * NQ);
        double bb = 0.0, gb = 0.0, bg = 0.0;
        for (int b = 0; b < P; ++b) {
          double tb = TB[(fz * P + b) * NQ + x_], tg = TG[(fz * P + b) * NQ + x_];
          bb += Bs[y_ * P + b] * tb;
          gb += Bs[y_ * P + b] * tg;
          bg += Gs[y_ * P + b] * tb;
        }
        PBB[w] = bb;
        PGB[w] = gb;
        PBG[w] = bg;
      }
    team_sync<NQD>();
    if (active)
      for (int f = 0; f < nf; ++f) {
        double d0 = 0.0, d1 = 0.0, d2 = 0.0;
        for (int cz = 0; cz < P; ++cz) {
          int idx = ((f * P + cz) * NQ + qy) * NQ + qx;
          d0 += Bs[qz * P + cz] * PGB[idx];
          d1 += Bs[qz * P + cz] * PBG[idx];
          d2 += Gs[qz * P + cz] * PBB[idx];
        }
        grad[f][0] = d0;
        grad[f][1] = d1;
        grad[f][2] = d2;
      }
  }
}

// out[j] (+)= sum_q phi_j(q) gq(q) over the team's quadrature points.
template <int DIM, int K, int NQD>
__device__ __forceinline__ void l2_contract(const double* gq, double* l2s, const double* Ls,
                                            int tq, bool active, double* out, bool add) {
  constexpr int NQ = 2 * K, ND2 = ipow(K, DIM);
  if constexpr (DIM == 2) {
    if (active)
      for (int w = tq; w < K * NQ; w += NQD) {
        int y_ = w % NQ, jx = w / NQ;
        double s = 0.0;
        for (int x_ = 0; x_ < NQ; ++x_) s += Ls[x_ * K + jx] * gq[y_ * NQ + x_];
        l2s[w] = s;
      }
    team_sync<NQD>();
    if (active)
      for (int j = tq; j < ND2; j += NQD) {
        int jx = j % K, jy = j / K;
        double s = 0.0;
        for (int y_ = 0; y_ < NQ; ++y_) s += Ls[y_ * K + jy] * l2s[jx * NQ + y_];
        out[j] = add ? out[j] + s : s;
      }
  } else {
    double* R1 = l2s;
    double* R2 = l2s + K * NQ * NQ;
    if (active)
      for (int w = tq; w < K * NQ * NQ; w += NQD) {
        int y_ = w % NQ, z_ = (w / NQ) % NQ, jx = w / (NQ * NQ);
        double s = 0.0;
        for (int x_ = 0; x_ < NQ; ++x_) s += Ls[x_ * K + jx] * gq[(z_ * NQ + y_) * NQ + x_];
        R1[w] = s;
      }
    team_sync<NQD>();
    if (active)
      for (int w = tq; w < K * K * NQ; w += NQD) {
        int z_ = w % NQ, jx = (w / NQ) % K, jy = w / (NQ * K);
        double s = 0.0;
        for (int y_ = 0; y_ < NQ; ++y_) s += Ls[y_ * K + jy] * R1[(jx * NQ + z_) * NQ + y_];
        R2[w] = s;
      }
    team_sync<NQD>();
    if (active)
      for (int j = tq; j < ND2; j += NQD) {
        int jx = j % K, jy = (j / K) % K, jz = j / (K * K);
        double s = 0.0;
        for (int z_ = 0; z_ < NQ; ++z_) s += Ls[z_ * K + jz] * R2[(jy * K + jx) * NQ + z_];
        out[j] = add ? out[j] + s : s;
      }
  }
}

// One tile of EPB elements [el0, el0 + EPB) of the energy update.  Every
// thread of the block calls it (it synchronises the block).
template <int DIM, int K, bool MIXED, int NTT>
__device__ __forceinline__ void energy_tile(const Geom& g, const Basis1D& bas, const EnergyArgs& A,
                                            const double* rho0Kp, unsigned char* smem,
                                            int64_t el0) {
  using F = EL<DIM, K, MIXED, NTT>;
  constexpr int P = F::P, NQ = F::NQ, ND1 = F::ND1, ND2 = F::ND2, NQD = F::NQD;
  const double coef = A.rate ? A.frac : A.frac * (A.ctl != nullptr ? A.ctl->dt_use : A.dt);
  // mixed path: F^T w of the reference pressure -p_ref I, in FP64
  const double pref = (MIXED && A.p_ref != nullptr && A.x != nullptr) ? *A.p_ref : 0.0;
  unsigned char* sp = smem;
  double* Bs = reinterpret_cast<double*>(sp); sp += F::al(NQ * P * 8);
  double* Gs = reinterpret_cast<double*>(sp); sp += F::al(NQ * P * 8);
  double* Wd = reinterpret_cast<double*>(sp); sp += F::al(NQ * P * 8);
  double* Ls = reinterpret_cast<double*>(sp); sp += F::al(NQ * K * 8);
  double* Mi = reinterpret_cast<double*>(sp); sp += F::al(81 * 8);
  unsigned char* const area = sp;  // element areas, B_ELEM bytes each
  constexpr size_t O_SCR = F::al(F::NFI * ND1 * 8);
  constexpr size_t O_GQ = O_SCR + F::al(F::S_INTERP * 8);
  constexpr size_t O_L2 = O_GQ + F::al(NQD * 8);
  constexpr size_t O_FTV = O_L2 + F::al(F::S_L2 * 8);
  constexpr size_t O_PART = O_FTV + F::al(ND2 * 8);
  constexpr size_t O_FTVP = O_PART + F::al(NQD * 8);
  const int tid = threadIdx.x, le = tid / NQD, tq = tid - le * NQD;
  unsigned char* ep = area + le * F::B_ELEM;
  double* ws = reinterpret_cast<double*>(ep);  // w, then x
  double* scr = reinterpret_cast<double*>(ep + O_SCR);
  double* gq = reinterpret_cast<double*>(ep + O_GQ);
  double* l2s = reinterpret_cast<double*>(ep + O_L2);
  double* ftv = reinterpret_cast<double*>(ep + O_FTV);

  // slot el0 + le: the element itself, or (list mode) the listed element
  const int64_t nslots = A.list ? A.nslots : g.nelem;
  const int64_t slot = el0 + le;
  const bool active = le < F::EPB && slot < nslots;
  const int64_t el = active ? (A.list ? (int64_t)A.list[slot] : slot) : 0;
  int E[3] = {0, 0, 0};
  elem_ijk(g, el, E);
  // the (element, row) pair this thread updates at the end of the tile
  // (EPB ND2 = NTT / 2^DIM pairs): its loads are issued now
  static_assert(F::EPB * ND2 <= NTT, "one (element, row) pair per thread");
  const int lo = tid / ND2, jo = tid - lo * ND2;
  const bool out = tid < F::EPB * ND2 && el0 + lo < nslots;
  double eb = 0.0, rk = 1.0;
  if (out && A.FTvE == nullptr) {
    if (!A.rate) eb = A.e_base[(el0 + lo) * ND2 + jo];
    rk = A.rho0Kinv ? A.rho0Kinv[el0 + lo] : rho0Kp[el0 + lo];
  }

  if constexpr (MIXED) {
    // F^T w from the stored FP32 element matrix, to ~2^-48: w is split into
    // two floats, each product f w_hi is formed exactly (TwoProduct), the
    // terms are added with error-free sums and the errors collected apart,
    // all on the FP32 pipe.  The team's NQD = 2^DIM ND2 threads split the
    // DIM ND1 terms of each of the ND2 sums into 2^DIM chunks (thread tq:
    // row j = tq mod ND2, chunk tq / ND2); each thread loads its chunk's
    // matrix entries and w values itself, every load issued before the
    // first use.  The chunk sums are added in chunk order below.
    constexpr int NPART = NQD / ND2, NCI = DIM * ND1, CH = (NCI + NPART - 1) / NPART;
    constexpr int UB = CH < 6 ? CH : 6;  // loads in flight per batch
    float2* part = reinterpret_cast<float2*>(ep + O_PART);
    const int j = tq % ND2, pc = tq / ND2;
    const int c0 = pc * CH, c1 = (c0 + CH < NCI) ? c0 + CH : NCI;
    float S = 0.0f, C = 0.0f;
    if (active) {
      const float* fk = A.FK + el * (DIM * ND1 * ND2);
      for (int u0 = c0; u0 < c1; u0 += UB) {
        float fv[UB];
        double wv[UB];
#pragma unroll
        for (int u = 0; u < UB; ++u) {
          const int ci = u0 + u;
          fv[u] = 0.0f;
          wv[u] = 0.0;
          if (ci < c1) {
            const int c = ci / ND1, i = ci - c * ND1;
            const int a = i % P, b = (i / P) % P, cc = DIM == 3 ? i / (P * P) : 0;
            fv[u] = fk[ci * ND2 + j];
            wv[u] = A.w[c * g.nnodes + elem_node<K>(g, E, a, b, cc)];
          }
        }
#pragma unroll
        for (int u = 0; u < UB; ++u) {
          if (u0 + u >= c1) break;
          float wh, wl;
          split_df(wv[u], wh, wl);
          const float f = fv[u];
          const float p = __fmul_rn(f, wh);
          const float pe = __fmaf_rn(f, wh, -p);  // f w_hi - p, exact
          float s2, e2;
          two_sum_f(S, p, s2, e2);
          S = s2;
          C = __fadd_rn(C, __fadd_rn(e2, __fmaf_rn(f, wl, pe)));
        }
      }
      part[tq] = make_float2(S, C);
    }
    if (pref != 0.0) {
      // -p_ref alpha_q tr(adj(J) grad w) at the points, J from the FP64
      // positions, contracted into ftvp
      if (active) {
        constexpr int PS = (2 * DIM * ND1 + NQD - 1) / NQD;
        double sv[PS];
#pragma unroll
        for (int jj = 0; jj < PS; ++jj) {
          const int w = tq + jj * NQD;
          sv[jj] = 0.0;
          if (w < 2 * DIM * ND1) {
            const int f = w / ND1, i = w - f * ND1;
            const int a = i % P, b = (i / P) % P, cc = DIM == 3 ? i / (P * P) : 0;
            const int64_t node = elem_node<K>(g, E, a, b, cc);
            sv[jj] = f < DIM ? A.w[f * g.nnodes + node] : A.x[(f - DIM) * g.nnodes + node];
          }
        }
#pragma unroll
        for (int jj = 0; jj < PS; ++jj)
          if (tq + jj * NQD < 2 * DIM * ND1) ws[tq + jj * NQD] = sv[jj];
      }
      team_sync<NQD>();
      double grad[2 * DIM][DIM];
      interp_grads<DIM, K, NQD, 2 * DIM>(ws, 2 * DIM, scr, Bs, Gs, tq, active, grad);
      if (active) {
        const int qx = tq % NQ, qy = (tq / NQ) % NQ, qz = DIM == 3 ? tq / (NQ * NQ) : 0;
        double J[DIM][DIM], Aj[DIM][DIM];
        for (int c = 0; c < DIM; ++c)
          for (int m = 0; m < DIM; ++m) J[c][m] = grad[DIM + c][m];
        adj_of<double, DIM>(J, Aj);
        double tr = 0.0;
        for (int c = 0; c < DIM; ++c)
          for (int m = 0; m < DIM; ++m) tr += Aj[m][c] * grad[c][m];
        const double alpha = Wd[qx] * Wd[qy] * (DIM == 3 ? Wd[qz] : 1.0);
        gq[tq] = -pref * alpha * tr;
      }
      team_sync<NQD>();
      l2_contract<DIM, K, NQD>(gq, l2s, Ls, tq, active,
                               reinterpret_cast<double*>(ep + O_FTVP), false);
    }
    __syncthreads();
    // F^T w rows: the chunk sums of row j in chunk order, widened to FP64
    for (int idx = tid; idx < F::EPB * ND2; idx += NTT) {
      const int l = idx / ND2, jr = idx - l * ND2;
      if (el0 + l >= nslots) continue;
      const unsigned char* e2p = area + l * F::B_ELEM;
      const float2* pp = reinterpret_cast<const float2*>(e2p + O_PART);
      float S2 = pp[jr].x, C2 = pp[jr].y;
      for (int q = 1; q < NPART; ++q) {
        const float2 r = pp[q * ND2 + jr];
        float s2, e2;
        two_sum_f(S2, r.x, s2, e2);
        S2 = s2;
        C2 = __fadd_rn(C2, __fadd_rn(e2, r.y));
      }
      double f = f2d_exact(S2) + f2d_exact(C2);
      if (pref != 0.0) f += reinterpret_cast<const double*>(e2p + O_FTVP)[jr];
      reinterpret_cast<double*>(area + l * F::B_ELEM + O_FTV)[jr] = f;
    }
  } else {
    if (active) {  // loads first, then the shared-memory stores
      constexpr int PS = (DIM * ND1 + NQD - 1) / NQD;
      double sv[PS];
#pragma unroll
      for (int jj = 0; jj < PS; ++jj) {
        const int w = tq + jj * NQD;
        sv[jj] = 0.0;
        if (w < DIM * ND1) {
          const int f = w / ND1, i = w - f * ND1;
          const int a = i % P, b = (i / P) % P, cc = DIM == 3 ? i / (P * P) : 0;
          sv[jj] = A.w[f * g.nnodes + elem_node<K>(g, E, a, b, cc)];
        }
      }
#pragma unroll
      for (int jj = 0; jj < PS; ++jj)
        if (tq + jj * NQD < DIM * ND1) ws[tq + jj * NQD] = sv[jj];
    }
    team_sync<NQD>();
    double gw[DIM][DIM];
    interp_grads<DIM, K, NQD, DIM>(ws, DIM, scr, Bs, Gs, tq, active, gw);
    if (active) {
      const double* D = A.D + el * DIM * DIM * NQD;
      double s = 0.0;
      for (int c = 0; c < DIM; ++c)
        for (int m = 0; m < DIM; ++m) s += D[(c * DIM + m) * NQD + tq] * gw[c][m];
      gq[tq] = s;
    }
    team_sync<NQD>();
    l2_contract<DIM, K, NQD>(gq, l2s, Ls, tq, active, ftv, false);
  }
  __syncthreads();
  // per (element, row) of the tile: the F^T w rows (list mode), or
  // e_out = e_base + coef M_E,K^{-1} (F^T w + src) with
  // M_E,K^{-1} = Mref^{-1} / (rho0 |J0|)_K
  if (out) {
    const int64_t sl = el0 + lo;
    const double* fv = reinterpret_cast<const double*>(area + lo * F::B_ELEM + O_FTV);
    if (A.FTvE != nullptr) {
      A.FTvE[sl * ND2 + jo] = fv[jo];
    } else {
      const double crs = A.rho0Kinv ? coef * rk : coef / rk;
      double s = 0.0;
      for (int q = 0; q < ND2; ++q) {
        double rhs = fv[q];
        if (A.srcE) rhs += A.srcE[sl * ND2 + q];
        s = fma(Mi[jo * ND2 + q], rhs, s);
      }
      A.e_out[sl * ND2 + jo] = A.rate ? crs * s : fma(crs, s, eb);
    }
  }
  __syncthreads();  // the element areas are reused by the next tile
}

template <int DIM, int K, bool MIXED>
__global__ void __launch_bounds__(EL<DIM, K, MIXED>::NT)
energy_update_kernel(const EnergyKParams prm) {
  pdl_enter();
  using F = EL<DIM, K, MIXED>;
  if (prm.a.ctl != nullptr && prm.a.ctl->done) return;
  extern __shared__ __align__(16) unsigned char smem[];
  energy_tables<DIM, K, MIXED, F::NT>(prm.b, smem);
  __syncthreads();
  energy_tile<DIM, K, MIXED, F::NT>(prm.g, prm.b, prm.a, prm.rho0K, smem,
                                    (int64_t)blockIdx.x * F::EPB);
}

}  // namespace lagh
