// Element operator of the partially assembled kinematic mass matrix, shared by
// the mass-apply kernel and the CG kernels.
#pragma once

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
    for (int a = 0; a < P; ++a) s = fma(M1[ap * P + a], u[base + a], s);
    t[w] = s;
  }
  __syncthreads();
  if constexpr (DIM == 2) {
    for (int w = threadIdx.x; w < items; w += blockDim.x) {
      int i = w % ND1, base = w - i, a = i % P, bp = i / P;
      double s = 0.0;
      for (int b = 0; b < P; ++b) s = fma(M1[bp * P + b], t[base + b * P + a], s);
      y[w] = s;
    }
  } else {
    for (int w = threadIdx.x; w < items; w += blockDim.x) {
      int i = w % ND1, base = w - i, a = i % P, bp = (i / P) % P, cz = i / (P * P);
      double s = 0.0;
      for (int b = 0; b < P; ++b) s = fma(M1[bp * P + b], t[base + (cz * P + b) * P + a], s);
      u[w] = s;  // u is free again
    }
    __syncthreads();
    for (int w = threadIdx.x; w < items; w += blockDim.x) {
      int i = w % ND1, base = w - i, ab = i % (P * P), czp = i / (P * P);
      double s = 0.0;
      for (int cz = 0; cz < P; ++cz) s = fma(M1[czp * P + cz], u[base + cz * P * P + ab], s);
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

}  // namespace lagh
