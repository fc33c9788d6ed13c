// Device helpers shared by the kernels of the library: structured-mesh index
// arithmetic, deterministic block reductions, the ordered-bits minimum used for
// the time-step estimate and a bounded grid barrier for cooperative kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lagh_impl.cuh"

namespace lagh {

// ---------------------------------------------------------------- mesh ----

// Node multi-index (I, J, K) of a lexicographic node number.
__device__ __forceinline__ void node_ijk(const Geom& g, int64_t node, int I[3]) {
  I[0] = (int)(node % g.nn[0]);
  int64_t r = node / g.nn[0];
  I[1] = (int)(r % g.nn[1]);
  I[2] = (int)(r / g.nn[1]);
}

__device__ __forceinline__ int64_t node_index(const Geom& g, int I, int J, int K3) {
  return (int64_t)I + (int64_t)g.nn[0] * ((int64_t)J + (int64_t)g.nn[1] * K3);
}

// Element multi-index of a lexicographic element number.
__device__ __forceinline__ void elem_ijk(const Geom& g, int64_t el, int E[3]) {
  E[0] = (int)(el % g.n[0]);
  int64_t r = el / g.n[0];
  E[1] = (int)(r % g.n[1]);
  E[2] = (int)(r / g.n[1]);
}

// Global node of local node (a, b, c) of element (E0, E1, E2).
template <int K>
__device__ __forceinline__ int64_t elem_node(const Geom& g, const int E[3], int a, int b, int cc) {
  return node_index(g, E[0] * K + a, E[1] * K + b, E[2] * K + cc);
}

// Wall condition: component c of a node on a face x_c = lo_c or hi_c.
__device__ __forceinline__ bool essential(const Geom& g, const int I[3], int c) {
  return I[c] == 0 || I[c] == g.nn[c] - 1;
}

// The (at most two) elements along one direction that contain node index I,
// with the local node index inside each, in increasing element order.
template <int K>
__device__ __forceinline__ int node_elems_1d(int I, int nel, int* el, int* loc) {
  int cnt = 0;
  int q = I / K, r = I - q * K;
  if (r == 0) {
    if (q > 0) { el[cnt] = q - 1; loc[cnt] = K; ++cnt; }
    if (q < nel) { el[cnt] = q; loc[cnt] = 0; ++cnt; }
  } else {
    el[cnt] = q; loc[cnt] = r; ++cnt;
  }
  return cnt;
}

// Deterministic gather of an element-local kinematic vector E[el][c][i] at one
// node: the contributions of the <= 2^DIM elements are summed in a fixed order.
template <int DIM, int K>
__device__ __forceinline__ double gather_node(const Geom& g, const double* __restrict__ E,
                                              const int I[3], int c) {
  constexpr int P = K + 1;
  constexpr int ND1 = DIM == 2 ? P * P : P * P * P;
  int ex[2], lx[2], ey[2], ly[2], ez[2] = {0, 0}, lz[2] = {0, 0};
  int nx = node_elems_1d<K>(I[0], g.n[0], ex, lx);
  int ny = node_elems_1d<K>(I[1], g.n[1], ey, ly);
  int nz = 1;
  if (DIM == 3) nz = node_elems_1d<K>(I[2], g.n[2], ez, lz);
  double s = 0.0;
  for (int kz = 0; kz < nz; ++kz)
    for (int ky = 0; ky < ny; ++ky)
      for (int kx = 0; kx < nx; ++kx) {
        int64_t el = (int64_t)ex[kx] + (int64_t)g.n[0] * ((int64_t)ey[ky] + (int64_t)g.n[1] * ez[kz]);
        int i = lx[kx] + P * (ly[ky] + P * lz[kz]);
        s += E[(el * DIM + c) * ND1 + i];
      }
  return s;
}

// ---------------------------------------------------------- reductions ----

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Block sum in a fixed order (lane tree, then warps in order).  All threads
// must call it; the result is valid in thread 0.  sh: >= 32 doubles.
__device__ __forceinline__ double block_sum(double v, double* sh) {
  v = warp_sum(v);
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0) {
    int nw = (blockDim.x + 31) >> 5;
    for (int i = 0; i < nw; ++i) s += sh[i];
  }
  return s;
}

// Non-negative doubles order like their bit patterns; +inf is the identity.
__device__ __forceinline__ unsigned long long tau_to_bits(double t) {
  if (!(t >= 0.0)) t = 0.0;  // NaN or negative: force a redo
  return (unsigned long long)__double_as_longlong(t);
}

__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long v) {
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long w = __shfl_down_sync(0xffffffffu, v, o);
    v = w < v ? w : v;
  }
  return v;
}

// Block minimum of the ordered bits, then one atomicMin per block (min is
// exact and order-independent, so the result is deterministic).  Works for
// any block size (a shared-memory tree, no partial-warp shuffles).
// sh: >= blockDim.x entries; blockDim.x <= 1024.
__device__ __forceinline__ void block_min_to(unsigned long long v, unsigned long long* sh,
                                             unsigned long long* dst) {
  const int tid = threadIdx.x, n = blockDim.x;
  __syncthreads();
  sh[tid] = v;
  __syncthreads();
  for (int s = 512; s > 0; s >>= 1) {
    if (tid < s && tid + s < n) {
      unsigned long long w = sh[tid + s];
      if (w < sh[tid]) sh[tid] = w;
    }
    __syncthreads();
  }
  if (tid == 0) atomicMin(dst, sh[0]);
}

// ------------------------------------------------------------- barrier ----

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier for a cooperative launch (all blocks co-resident).  The
// wait is bounded: after ~2 s it records kDevTimeout in *status and returns
// false, so the kernel can leave instead of hanging.
__device__ __forceinline__ bool grid_barrier(Barrier* bar, int* status) {
  __shared__ int ok_sh;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int* vgen = &bar->gen;
    unsigned int gen = *vgen;
    __threadfence();
    unsigned int arrived = atomicAdd(&bar->count, 1u);
    int ok = 1;
    if (arrived == gridDim.x - 1) {
      atomicExch(&bar->count, 0u);
      __threadfence();
      atomicAdd(&bar->gen, 1u);
    } else {
      unsigned long long t0 = global_ns();
      while (*vgen == gen) {
        __nanosleep(40);
        if (global_ns() - t0 > 2000000000ull) {
          atomicOr(status, kDevTimeout);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
    ok_sh = ok;
  }
  __syncthreads();
  return ok_sh != 0;
}

}  // namespace lagh
