// Device helpers shared by the kernels of the library: structured-mesh index
// arithmetic, deterministic block reductions, the ordered-bits minimum used for
// the time-step estimate, integer-pipe precision conversions and dependent
// launches.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lagh_impl.cuh"

namespace lagh {

// ------------------------------------------------- dependent launches ----
// Programmatic dependent launch: a kernel launched with the programmatic
// stream-serialisation attribute may be launched while its predecessor
// drains; it waits here (in hardware) until the predecessor has completed and
// its memory is visible.  Without the attribute it is a no-op.  Every kernel
// of the step calls pdl_enter() before touching memory.  An explicit early
// trigger (pdl_launch_dependents) was measured slower on the 64x64 step (the
// waiting successor's blocks compete with the running grid), so the trigger
// stays implicit at grid completion.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_dependents() {
  asm volatile("griddepcontrol.launch_dependents;" :::);
}
__device__ __forceinline__ void pdl_enter() { pdl_wait(); }

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
// node: the contributions of the <= 2^DIM elements are summed in a fixed order
// (the first one starts the sum; every node lies in at least one element).
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
  double v[DIM == 3 ? 8 : 4];
#pragma unroll
  for (int kz = 0; kz < (DIM == 3 ? 2 : 1); ++kz)
#pragma unroll
    for (int ky = 0; ky < 2; ++ky)
#pragma unroll
      for (int kx = 0; kx < 2; ++kx) {
        const int t = (kz * 2 + ky) * 2 + kx;
        v[t] = 0.0;
        if (kx < nx && ky < ny && kz < nz) {
          int64_t el = (int64_t)ex[kx] + (int64_t)g.n[0] * ((int64_t)ey[ky] + (int64_t)g.n[1] * ez[kz]);
          int i = lx[kx] + P * (ly[ky] + P * lz[kz]);
          v[t] = E[(el * DIM + c) * ND1 + i];
        }
      }
  double s = v[0];
#pragma unroll
  for (int kz = 0; kz < (DIM == 3 ? 2 : 1); ++kz)
#pragma unroll
    for (int ky = 0; ky < 2; ++ky)
#pragma unroll
      for (int kx = 0; kx < 2; ++kx) {
        const int t = (kz * 2 + ky) * 2 + kx;
        if (t > 0 && kx < nx && ky < ny && kz < nz) s += v[t];
      }
  return s;
}

// ------------------------------------------------ precision conversions ----
// On this GPU FP64 arithmetic issues at 1/64 of the FP32 rate, and the FP64
// pipe also executes conversions between FP32 and FP64.  The FP32 paths
// therefore convert with integer operations (IEEE 754 bit layouts: FP32 has an
// 8-bit exponent biased by 127 and a 23-bit fraction, FP64 an 11-bit exponent
// biased by 1023 and a 52-bit fraction).

// Exact FP32 -> FP64 (every float is a double): rebias the exponent, widen the
// fraction; subnormal floats are normalised, inf / NaN keep their class.
__device__ __forceinline__ double f2d_exact(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned long long s = (unsigned long long)(u & 0x80000000u) << 32;
  const unsigned ex = (u >> 23) & 0xffu;
  const unsigned m = u & 0x7fffffu;
  unsigned long long bits;
  if (ex == 0u) {
    if (m == 0u) {
      bits = s;
    } else {  // m 2^-149 with its leading bit at position p
      const int p = 31 - __clz((int)m);
      bits = s | ((unsigned long long)(p + 874) << 52) |
             (((unsigned long long)m << (52 - p)) & 0xfffffffffffffull);
    }
  } else if (ex == 0xffu) {
    bits = s | 0x7ff0000000000000ull | ((unsigned long long)m << 29);
  } else {
    bits = s | ((unsigned long long)(ex + 896u) << 52) | ((unsigned long long)m << 29);
  }
  return __longlong_as_double((long long)bits);
}

// FP64 -> FP32 rounded to nearest, ties to even (as a C cast), with integer
// operations only: results in the FP32 subnormal range are rounded to its
// 2^-149 grid, results above the range round to infinity, NaN stays NaN.
__device__ __forceinline__ float d2f_rn(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const unsigned s = (unsigned)(b >> 32) & 0x80000000u;
  const int ex = (int)((b >> 52) & 0x7ffu);
  const unsigned long long m = b & 0xfffffffffffffull;
  if (ex == 0x7ff) return __uint_as_float(s | 0x7f800000u | (m ? 0x400000u : 0u));
  int fe = ex - 896;  // FP32 biased exponent
  if (fe <= 0) {  // subnormal result: the 53-bit significand in units of 2^-149
    const int sh = 30 - fe;
    if (ex == 0 || sh > 54) return __uint_as_float(s);  // below half of 2^-149
    const unsigned long long M = m | (1ull << 52);
    unsigned r = (unsigned)(M >> sh);
    const unsigned long long rem = M & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
    if (rem > half || (rem == half && (r & 1u))) ++r;  // may carry into 2^-126
    return __uint_as_float(s | r);
  }
  unsigned r = (unsigned)(m >> 29);
  const unsigned rem = (unsigned)(m & 0x1fffffffull);
  if (rem > 0x10000000u || (rem == 0x10000000u && (r & 1u))) {
    if (++r == 0x800000u) {  // the fraction carried into the exponent
      r = 0u;
      ++fe;
    }
  }
  if (fe >= 0xff) return __uint_as_float(s | 0x7f800000u);
  return __uint_as_float(s | ((unsigned)fe << 23) | r);
}

// Error-free transformations in FP32 (two-float "double-float" sums): with
// the rounding-exact intrinsics the compiler neither fuses nor reorders them.
// two_sum_f: s + e == a + b exactly (s = fl(a + b)).
__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// w = hi + lo to about 2^-48 relative: hi is w with its 29 lowest fraction
// bits cleared (exactly a float), lo the cleared part rounded to a float.
// Integer operations only; |w| below 2^-75 or outside the FP32 range keeps
// lo = 0 (then hi carries the FP32 rounding of w, or 0 / inf).
__device__ __forceinline__ void split_df(double w, float& hi, float& lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(w);
  hi = d2f_rn(__longlong_as_double((long long)(b & ~0x1fffffffull)));
  const int ex = (int)((b >> 52) & 0x7ffu);
  const unsigned low = (unsigned)(b & 0x1fffffffull);
  const int fe = ex - 948;  // FP32 biased exponent of 2^(ex - 1075)
  if (low == 0u || fe <= 0 || fe >= 0xff || ex == 0x7ff || hi == 0.0f) {
    lo = 0.0f;
    return;
  }
  const float l = __fmul_rn(__uint2float_rn(low), __uint_as_float((unsigned)fe << 23));
  lo = (b >> 63) ? -l : l;
}

template <typename T>
__device__ __forceinline__ T from_double(double d);
template <>
__device__ __forceinline__ double from_double<double>(double d) { return d; }
template <>
__device__ __forceinline__ float from_double<float>(double d) { return d2f_rn(d); }

__device__ __forceinline__ double to_double(double d) { return d; }
__device__ __forceinline__ double to_double(float f) { return f2d_exact(f); }

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

}  // namespace lagh
