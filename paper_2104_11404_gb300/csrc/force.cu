// Force kernels of the Lagrangian step: the generalized force matrix F of
// eq:fom applied matrix-free as F.1 and F^T.v (eq:forceOneforceTv) with sum
// factorisation over the tensor-product element.
//
// One CTA processes EPB elements; each element is owned by a team of NQ^DIM
// threads (one per quadrature point).  Element data are staged in shared
// memory, the reference gradients at the quadrature points are built in
// DIM passes of 1D contractions, the stress is formed per point, and the
// transposed contractions return the element rows of F.1.  Element rows go
// to an element-local array; a node-wise gather sums them in a fixed order
// (no floating-point atomics).
//
// FP64 path: the per-point stress weights D_q = alpha_q sigma_q adj(J_q)^T are
//   kept (double) for the later F^T.v of the same stage.
// Mixed path: stress in FP32; the element matrix F_K[(c,i), j] is assembled in
//   FP32 and kept; F.1 (row sums) and F^T.v are FP64 contractions of those
//   FP32 entries, so v.(F.1) = 1.(F^T v) holds to FP64 rounding and the
//   RK2-average energy balance stays exact.
#include "force_tiles.cuh"

namespace lagh {

// ---------------------------------------------------------- launchers ----

template <int DIM, int K, bool MIXED>
static cudaError_t launch_force_t(const lh_ctx* c, const ForceArgs& fa, cudaStream_t s) {
  using F = FL<DIM, K, MIXED>;
  using F1 = FL<DIM, K, MIXED, F::TEAM>;  // one element per block
  if (fa.nslots == 0) return cudaSuccess;
  ForceKParams prm;
  prm.g = c->g;
  prm.ph = c->ph;
  prm.b = c->basis;
  prm.a = fa;
  prm.a.gammaE = c->a.gammaE;
  prm.rho0K = c->a.rho0K;
  int64_t blocks = (fa.nslots + F::EPB - 1) / F::EPB;
  // a short element list (a sampled subset) would leave most SMs idle with
  // several elements per block: one element per block spreads it out (each
  // element's arithmetic is the same either way).  Only for teams of whole
  // warps (3D Q2: 64 threads), so every warp-level primitive sees full warps.
  if constexpr (F::TEAM % 32 == 0) {
    if (fa.list != nullptr && F::EPB > 1 && blocks < c->num_sms)
      return launch_k(c->use_pdl != 0, force_kernel<DIM, K, MIXED, F::TEAM>,
                      dim3((unsigned)fa.nslots), dim3(F1::NT), F1::BYTES, s, prm);
  }
  return launch_k(c->use_pdl != 0, force_kernel<DIM, K, MIXED>, dim3((unsigned)blocks),
                  dim3(F::NT), F::BYTES, s, prm);
}

#define LAGH_DISPATCH(DIMV, KV, FN, ...)                                            \
  do {                                                                              \
    if ((DIMV) == 2 && (KV) == 1) return FN<2, 1>(__VA_ARGS__);                     \
    if ((DIMV) == 2 && (KV) == 2) return FN<2, 2>(__VA_ARGS__);                     \
    if ((DIMV) == 2 && (KV) == 3) return FN<2, 3>(__VA_ARGS__);                     \
    if ((DIMV) == 3 && (KV) == 1) return FN<3, 1>(__VA_ARGS__);                     \
    if ((DIMV) == 3 && (KV) == 2) return FN<3, 2>(__VA_ARGS__);                     \
    return cudaErrorInvalidValue;                                                   \
  } while (0)

template <int DIM, int K>
static cudaError_t launch_force_dk(const lh_ctx* c, const ForceArgs& fa, cudaStream_t s) {
  if (c->precision == LH_MIXED) return launch_force_t<DIM, K, true>(c, fa, s);
  return launch_force_t<DIM, K, false>(c, fa, s);
}

cudaError_t launch_force(const lh_ctx* c, const ForceArgs& fa, cudaStream_t s) {
  LAGH_DISPATCH(c->g.dim, c->g.k, launch_force_dk, c, fa, s);
}

template <int DIM, int K>
static cudaError_t launch_force64_dk(const lh_ctx* c, const ForceArgs& fa, cudaStream_t s) {
  return launch_force_t<DIM, K, false>(c, fa, s);
}

cudaError_t launch_force_fp64(const lh_ctx* c, const ForceArgs& fa, cudaStream_t s) {
  LAGH_DISPATCH(c->g.dim, c->g.k, launch_force64_dk, c, fa, s);
}

template <int DIM, int K>
static cudaError_t launch_gather_dk(const lh_ctx* c, const double* E, double* out, double scale,
                                    int apply_bc, const Ctl* ctl, cudaStream_t s) {
  const int nt = 256;
  int64_t blocks = (c->g.nnodes + nt - 1) / nt;
  return launch_k(c->use_pdl != 0, gather_kernel<DIM, K>, dim3((unsigned)blocks), dim3(nt), 0, s,
                  c->g, E, out, scale, apply_bc, ctl);
}

cudaError_t launch_gather(const lh_ctx* c, const double* E, double* out, double scale,
                          int apply_bc, const Ctl* ctl, cudaStream_t s) {
  LAGH_DISPATCH(c->g.dim, c->g.k, launch_gather_dk, c, E, out, scale, apply_bc, ctl, s);
}

template <int DIM, int K, bool MIXED>
static cudaError_t launch_energy_t(const lh_ctx* c, const EnergyArgs& ea, cudaStream_t s) {
  using F = EL<DIM, K, MIXED>;
  auto kern = energy_update_kernel<DIM, K, MIXED>;
  EnergyKParams prm;
  prm.g = c->g;
  prm.b = c->basis;
  prm.a = ea;
  prm.rho0K = c->a.rho0K;
  int64_t blocks = (c->g.nelem + F::EPB - 1) / F::EPB;
  return launch_k(c->use_pdl != 0, kern, dim3((unsigned)blocks), dim3(F::NT), F::BYTES, s, prm);
}

template <int DIM, int K, bool MIXED>
static cudaError_t launch_ftv_list_t(const lh_ctx* c, const EnergyArgs& ea, cudaStream_t s) {
  using F = EL<DIM, K, MIXED>;
  if (ea.nslots == 0) return cudaSuccess;
  EnergyKParams prm;
  prm.g = c->g;
  prm.b = c->basis;
  prm.a = ea;
  prm.rho0K = c->a.rho0K;
  int64_t blocks = (ea.nslots + F::EPB - 1) / F::EPB;
  return launch_k(c->use_pdl != 0, energy_update_kernel<DIM, K, MIXED>, dim3((unsigned)blocks),
                  dim3(F::NT), F::BYTES, s, prm);
}

template <int DIM, int K>
static cudaError_t launch_ftv_list_dk(const lh_ctx* c, const EnergyArgs& ea, cudaStream_t s) {
  if (c->precision == LH_MIXED) return launch_ftv_list_t<DIM, K, true>(c, ea, s);
  return launch_ftv_list_t<DIM, K, false>(c, ea, s);
}

cudaError_t launch_ftv_list(const lh_ctx* c, const EnergyArgs& ea, cudaStream_t s) {
  LAGH_DISPATCH(c->g.dim, c->g.k, launch_ftv_list_dk, c, ea, s);
}

template <int DIM, int K>
static cudaError_t launch_energy_dk(const lh_ctx* c, const EnergyArgs& ea, cudaStream_t s) {
  if (c->precision == LH_MIXED) return launch_energy_t<DIM, K, true>(c, ea, s);
  return launch_energy_t<DIM, K, false>(c, ea, s);
}

cudaError_t launch_energy_update(const lh_ctx* c, const EnergyArgs& ea, cudaStream_t s) {
  LAGH_DISPATCH(c->g.dim, c->g.k, launch_energy_dk, c, ea, s);
}

// Opt the kernels of this context's (dim, order, precision) into their
// dynamic shared memory before any stream capture.
template <int DIM, int K, bool MIXED>
static cudaError_t prepare_t() {
  cudaError_t e = cudaFuncSetAttribute(force_kernel<DIM, K, MIXED>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)FL<DIM, K, MIXED>::BYTES);
  if (e != cudaSuccess) return e;
  constexpr int TEAM = FL<DIM, K, MIXED>::TEAM;
  if constexpr (TEAM % 32 == 0) {
    e = cudaFuncSetAttribute(force_kernel<DIM, K, MIXED, TEAM>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)FL<DIM, K, MIXED, TEAM>::BYTES);
    if (e != cudaSuccess) return e;
  }
  return cudaFuncSetAttribute(energy_update_kernel<DIM, K, MIXED>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)EL<DIM, K, MIXED>::BYTES);
}

template <int DIM, int K>
static cudaError_t prepare_dk(const lh_ctx* c) {
  cudaError_t e = prepare_t<DIM, K, false>();  // FP64 kernels serve the mixed path too
  if (e != cudaSuccess || c->precision != LH_MIXED) return e;
  return prepare_t<DIM, K, true>();
}

cudaError_t prepare_kernels(const lh_ctx* c) { LAGH_DISPATCH(c->g.dim, c->g.k, prepare_dk, c); }

}  // namespace lagh
