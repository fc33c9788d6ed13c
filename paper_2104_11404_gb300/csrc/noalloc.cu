// lh_force_static: one FP64 force evaluation (F.1 with the wall condition and
// the time-step estimate) that allocates no memory.
//
// Some callers cannot allocate device memory: code that runs where the
// allocator is owned by someone else (inside a framework's memory pool or a
// plugin that must not call cudaMalloc), code that must never stall on an
// allocation in a latency-critical loop, and callers that budget every byte
// of the device up front.  They cannot create a context (lh_create allocates
// its work arrays), so this entry point needs none: the caller passes the
// descriptors, the state and the output, and the only working memory is the
// fixed-size array below, which every GPU that loads the library holds until
// the process exits.
#include <mutex>
#include <string.h>

#include "lagh_impl.cuh"

namespace lagh {

// Working memory of lh_force_static: 4 Mi doubles (32 MiB).
//   [0]                 time-step estimate (ordered bits)
//   [1]                 error flags (int)
//   [16, 16 + n_e)      rho0 |J0| per element
//   [16 + n_e, ...)     element rows of F.1, n_e * dim * (k+1)^dim doubles
constexpr int64_t kStaticScratchDoubles = int64_t(1) << 22;
static __device__ __align__(256) double g_force_scratch[kStaticScratchDoubles];

constexpr int kMaxDevices = 64;

// Per-device set-up: the device address of the array (a host-side name of a
// __device__ variable is not a device address) and the shared-memory opt-in of
// the force kernels.  Done once per device, with that device current.
static std::mutex g_setup_mu;
static double* g_scratch_ptr[kMaxDevices];
static unsigned g_prepared[kMaxDevices];  // bit (dim * 4 + order) set once prepared

__global__ void static_init_kernel(double* scratch, int64_t nelem, double rho0K) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) {
    reinterpret_cast<unsigned long long*>(scratch)[0] = 0x7ff0000000000000ull;  // +inf
    reinterpret_cast<int*>(scratch + 1)[0] = 0;
  }
  for (int64_t el = i; el < nelem; el += (int64_t)gridDim.x * blockDim.x) scratch[16 + el] = rho0K;
}

}  // namespace lagh

using namespace lagh;

extern "C" lh_status lh_force_static(const lh_mesh_desc* mesh, const lh_disc_desc* disc,
                                     const lh_phys_desc* phys, const double* v, const double* e,
                                     const double* x, double* F1, double* dt_est, void* stream) {
  if (!mesh || !disc || !phys || !v || !e || !x || !F1) return LH_EINVAL;
  // geometry of the Cartesian box (the same quantities lh_create derives)
  lh_ctx c;
  memset(&c.g, 0, sizeof(c.g));
  memset(&c.a, 0, sizeof(c.a));
  c.use_pdl = 0;
  c.cg_cluster = 0;
  c.cg_tiles = 0;
  {
    lh_status gs = make_geom(mesh, disc, &c.g, nullptr);
    if (gs != LH_OK) return gs;
  }
  if (!(phys->gamma > 1.0) || phys->problem < LH_SEDOV || phys->problem > LH_UNIFORM)
    return LH_EINVAL;
  const Geom& g = c.g;
  const int d = g.dim, k = g.k;
  int nd1 = 1;
  for (int i = 0; i < d; ++i) nd1 *= k + 1;
  const double vol = g.detJ0;
  // the array must hold the per-element quadrature data and the element rows
  if (16 + g.nelem * (1 + (int64_t)d * nd1) > kStaticScratchDoubles) return LH_ETOOLARGE;

  c.ph.gamma = phys->gamma;
  c.ph.cfl = phys->cfl;
  c.ph.cfl_mu = phys->cfl_mu;
  c.ph.q1 = phys->q1;
  c.ph.q2 = phys->q2;
  c.ph.visc = phys->visc;
  c.ph.problem = phys->problem;
  c.ph.source = 0;
  set_phys_floats(c.ph);
  c.precision = LH_FP64;
  build_basis(k, g.nq, d, &c.basis);

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LH_ECUDA;
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (g_scratch_ptr[dev] == nullptr) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_force_scratch) != cudaSuccess || p == nullptr)
        return LH_ECUDA;
      g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    const unsigned bit = 1u << (d * 4 + k);
    if (!(g_prepared[dev] & bit)) {
      if (prepare_kernels(&c) != cudaSuccess) return LH_ECUDA;
      g_prepared[dev] |= bit;
    }
    scratch = g_scratch_ptr[dev];
  }
  cudaStream_t s = (cudaStream_t)stream;
  c.a.rho0K = scratch + 16;  // rho0 = 1 in every problem: rho0 |J0| = |K0|
  double* F1E = scratch + 16 + g.nelem;
  unsigned long long* tau_bits = reinterpret_cast<unsigned long long*>(scratch);
  int* flags = reinterpret_cast<int*>(scratch + 1);

  const int64_t blocks = (g.nelem + 255) / 256;
  static_init_kernel<<<(unsigned)(blocks < 4096 ? blocks : 4096), 256, 0, s>>>(scratch, g.nelem,
                                                                             vol);
  if (cudaGetLastError() != cudaSuccess) return LH_ECUDA;
  ForceArgs f = {};
  f.v = v;
  f.e = e;
  f.x = x;
  f.nslots = g.nelem;
  f.F1E = F1E;
  f.tau_bits = tau_bits;
  f.status = flags;
  f.mode = kForceFull;
  if (launch_force(&c, f, s) != cudaSuccess) return LH_ECUDA;
  if (launch_gather(&c, F1E, F1, 1.0, 1, nullptr, s) != cudaSuccess) return LH_ECUDA;
  // The estimate and the state-check flags are read back on every call: with
  // no context there is no later call that could report a tangled or
  // non-finite state, so the call always synchronizes.
  double hb[2];
  if (cudaMemcpyAsync(hb, scratch, sizeof(hb), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return LH_ECUDA;
  if (dt_est) memcpy(dt_est, &hb[0], sizeof(double));
  int fl;
  memcpy(&fl, &hb[1], sizeof(int));
  if (fl & kDevNonFinite) return LH_ENONFINITE;
  if (fl & kDevTangled) return LH_ETANGLED;
  return LH_OK;
}
