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
// The velocity CG that uses this operator lives in cg.cu.
//
// M_E (thermodynamic, block diagonal) is applied as (rho0|J0|)_K^{-1} Mref^{-1}.
#include "mass_ops.cuh"

namespace lagh {

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

// ------------------------------------------------ conversion self-check ----

namespace lagh {
__global__ void convert_check_kernel(const double* in, int64_t n, float* f_out, double* d_out,
                                     double* split_out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float f = d2f_rn(in[i]);
    f_out[i] = f;
    d_out[i] = f2d_exact(f);
    if (split_out) {
      float hi, lo;
      split_df(in[i], hi, lo);
      split_out[i] = f2d_exact(hi) + f2d_exact(lo);
    }
  }
}
}  // namespace lagh

extern "C" lh_status lh_check_conversions(const double* in, int64_t n, float* f_out,
                                          double* d_out, double* split_out, void* stream) {
  if (n < 0 || (n > 0 && (!in || !f_out || !d_out))) return LH_EINVAL;
  if (n == 0) return LH_OK;
  const int64_t blocks = (n + 255) / 256;
  lagh::convert_check_kernel<<<(unsigned)(blocks < 1024 ? blocks : 1024), 256, 0,
                               (cudaStream_t)stream>>>(in, n, f_out, d_out, split_out);
  return cudaGetLastError() == cudaSuccess ? LH_OK : LH_ECUDA;
}
