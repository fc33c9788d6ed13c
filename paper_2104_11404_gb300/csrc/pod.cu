// Proper orthogonal decomposition of a snapshot matrix (Section 4, eq:SVD and
// eq:energy_criteria): the thin SVD of S - offset 1^T by one-sided (Hestenes)
// Jacobi, parallel over column pairs, and the basis size by the singular-value
// criterion.
//
// Jacobi sweeps use the round-robin ordering: with N = n rounded up to even
// and M = N - 1, round r pairs column M with column r and columns (r + p) mod
// M and (r - p) mod M for p = 1 .. N/2 - 1, so the N/2 pairs of a round are
// disjoint and every pair meets once per sweep.  One CTA per pair computes
// the three inner products (fixed-order block sums), the rotation that makes
// the pair orthogonal, and rotates both columns in place.  Sweeps repeat until
// no pair needed a rotation (|a_p . a_q| <= sqrt(m) 2^-52 |a_p| |a_q|, the
// rounding level of the inner product, or a column at the rounding level of
// the whole matrix).  The left singular vectors are the
// final columns divided by their norms; no right singular vectors are formed.
#include "lagh_impl.cuh"

namespace lagh {

constexpr int kPodThreads = 256;

// Fixed-order sum of one value per thread over the CTA (all threads get it).
__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    red[32] = s;
  }
  __syncthreads();
  return red[32];
}

__global__ void pod_center_kernel(const double* __restrict__ S, const double* __restrict__ off,
                                  int64_t m, int64_t n, double* __restrict__ A) {
  const int64_t total = m * n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x)
    A[i] = off ? S[i] - off[i % m] : S[i];
}

// sq[j] = |A_j|^2, one CTA per column.
__global__ void __launch_bounds__(kPodThreads) pod_colsq_kernel(const double* __restrict__ A,
                                                                int64_t m, double* __restrict__ sq) {
  __shared__ double red[33];
  const double* a = A + (int64_t)blockIdx.x * m;
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < m; i += blockDim.x) s = fma(a[i], a[i], s);
  s = block_sum(s, red);
  if (threadIdx.x == 0) sq[blockIdx.x] = s;
}

// scal[0] = |A|_F^2 (columns added in index order), scal[1] = the column floor.
__global__ void pod_floor_kernel(const double* sq, int64_t n, double* scal) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double f = 0.0;
  for (int64_t j = 0; j < n; ++j) f += sq[j];
  scal[0] = f;
  scal[1] = 1e-32 * f;
}

__global__ void __launch_bounds__(kPodThreads)
pod_round_kernel(double* __restrict__ A, int64_t m, int64_t n, int64_t N, int64_t r,
                 const double* __restrict__ scal, double tol, int* __restrict__ rotated) {
  __shared__ double red[33];
  const int64_t M = N - 1, p = blockIdx.x;
  int64_t a = p == 0 ? M : (r + p) % M;
  int64_t b = p == 0 ? r : (r - p + M) % M;
  if (a >= n || b >= n || a == b) return;
  if (a > b) { const int64_t t = a; a = b; b = t; }
  double* ap = A + a * m;
  double* aq = A + b * m;
  double sa = 0.0, sb = 0.0, sg = 0.0;
  for (int64_t i = threadIdx.x; i < m; i += blockDim.x) {
    const double u = ap[i], w = aq[i];
    sa = fma(u, u, sa);
    sb = fma(w, w, sb);
    sg = fma(u, w, sg);
  }
  const double alpha = block_sum(sa, red);
  const double beta = block_sum(sb, red);
  const double gamma = block_sum(sg, red);
  const double floor2 = scal[1];
  if (alpha <= floor2 || beta <= floor2) return;
  if (gamma == 0.0 || fabs(gamma) <= tol * sqrt(alpha * beta)) return;
  const double zeta = (beta - alpha) / (2.0 * gamma);
  const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
  const double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
  for (int64_t i = threadIdx.x; i < m; i += blockDim.x) {
    const double u = ap[i], w = aq[i];
    ap[i] = c * u - s * w;
    aq[i] = s * u + c * w;
  }
  if (threadIdx.x == 0) atomicOr(rotated, 1);
}

// Descending order of the column norms (stable), sorted singular values and
// the basis size of the criterion, one CTA.
__global__ void __launch_bounds__(kPodThreads)
pod_select_kernel(const double* __restrict__ sq, int64_t n, double eps, int64_t* __restrict__ order,
                  double* __restrict__ sg_sorted, double* __restrict__ scal) {
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
    const double sj = sqrt(sq[j]);
    int64_t rank = 0;
    for (int64_t l = 0; l < n; ++l) {
      const double sl = sqrt(sq[l]);
      rank += (sl > sj) || (sl == sj && l < j);
    }
    order[rank] = j;
    sg_sorted[rank] = sj;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double total = 0.0;
    for (int64_t j = 0; j < n; ++j) total += sqrt(sq[j]);
    int64_t k = n;
    double acc = 0.0;
    for (int64_t r = 0; r < n; ++r) {
      acc += sg_sorted[r];
      if (acc >= eps * total) { k = r + 1; break; }
    }
    scal[2] = total > 0.0 ? (double)k : 0.0;
  }
}

// U[:, r] = A[:, order[r]] / sigma_r (zero columns stay zero).
__global__ void pod_gather_kernel(const double* __restrict__ A, int64_t m,
                                  const int64_t* __restrict__ order,
                                  const double* __restrict__ sg_sorted, double* __restrict__ U) {
  const int64_t r = blockIdx.y;
  const int64_t j = order[r];
  const double s = sg_sorted[r];
  const double inv = s > 0.0 ? 1.0 / s : 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x)
    U[r * m + i] = s > 0.0 ? A[j * m + i] * inv : 0.0;
}

}  // namespace lagh

using namespace lagh;

extern "C" lh_status lh_pod(const double* S, int64_t m, int64_t n, const double* offset,
                            double eps, double* U, double* sigma, double* work, int64_t* k,
                            int32_t* sweeps, void* stream) {
  if (!S || !U || !sigma || !work || !k || m < 1 || n < 1 || n > 65535 || !(eps > 0.0) ||
      !(eps <= 1.0))
    return LH_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  double* A = work;
  double* sq = A + m * n;
  int64_t* order = reinterpret_cast<int64_t*>(sq + n);
  double* scal = sq + 2 * n;
  int* flag = reinterpret_cast<int*>(scal + 4);
  const int64_t total = m * n;
  int64_t cblocks = (total + 255) / 256;
  if (cblocks > 152 * 32) cblocks = 152 * 32;
  pod_center_kernel<<<(unsigned)cblocks, 256, 0, s>>>(S, offset, m, n, A);
  pod_colsq_kernel<<<(unsigned)n, kPodThreads, 0, s>>>(A, m, sq);
  pod_floor_kernel<<<1, 32, 0, s>>>(sq, n, scal);
  if (cudaGetLastError() != cudaSuccess) return LH_ECUDA;
  const int64_t N = (n + 1) / 2 * 2, M = N - 1;
  const int max_sweeps = 60;
  // orthogonality at the rounding level of an m-term inner product (a fixed
  // 1e-15 sits below it for long columns, and the sweeps then chase noise)
  const double tol = sqrt((double)m) * 2.220446049250313e-16;
  int sweep = 0, hflag = 1;
  for (sweep = 1; sweep <= max_sweeps && n > 1; ++sweep) {
    if (cudaMemsetAsync(flag, 0, sizeof(int), s) != cudaSuccess) return LH_ECUDA;
    for (int64_t r = 0; r < M; ++r)
      pod_round_kernel<<<(unsigned)(N / 2), kPodThreads, 0, s>>>(A, m, n, N, r, scal, tol, flag);
    if (cudaGetLastError() != cudaSuccess) return LH_ECUDA;
    if (cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return LH_ECUDA;
    if (!hflag) break;
  }
  if (n == 1) { sweep = 1; hflag = 0; }
  if (sweeps) *sweeps = sweep > max_sweeps ? max_sweeps : sweep;
  pod_colsq_kernel<<<(unsigned)n, kPodThreads, 0, s>>>(A, m, sq);
  pod_select_kernel<<<1, kPodThreads, 0, s>>>(sq, n, eps, order, sigma, scal);
  int64_t gx = (m + 255) / 256;
  if (gx > 64) gx = 64;
  pod_gather_kernel<<<dim3((unsigned)gx, (unsigned)n), 256, 0, s>>>(A, m, order, sigma, U);
  if (cudaGetLastError() != cudaSuccess) return LH_ECUDA;
  double kd = 0.0;
  if (cudaMemcpyAsync(&kd, scal + 2, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return LH_ECUDA;
  *k = (int64_t)kd;
  return hflag ? LH_ECG : LH_OK;
}
