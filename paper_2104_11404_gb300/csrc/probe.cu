// Peak arithmetic-rate probe: a measurement service of the library (the
// paper has no counterpart).  The roofline of the FP64- and FP32-pipe-bound
// kernels is quoted against the rate this kernel reaches on the same GPU:
// every thread runs eight independent chains of fused multiply-adds, enough
// resident warps to hide the FMA latency on every SM, and nothing else (no
// memory traffic inside the loop).
#include "lagh_impl.cuh"

namespace lagh {

// lanes: the chains run on the first `lanes` lanes of every warp (32: all).
template <typename T>
__global__ void __launch_bounds__(256) fma_probe_kernel(T* sink, int64_t iters, T a, T b,
                                                        int lanes) {
  T x0 = T(threadIdx.x) * T(1e-3), x1 = x0 + T(0.1), x2 = x0 + T(0.2), x3 = x0 + T(0.3);
  T x4 = x0 + T(0.4), x5 = x0 + T(0.5), x6 = x0 + T(0.6), x7 = x0 + T(0.7);
  if ((int)(threadIdx.x & 31u) < lanes)
    for (int64_t i = 0; i < iters; ++i) {
      x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
      x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
  const T s = ((x0 + x1) + (x2 + x3)) + ((x4 + x5) + (x6 + x7));
  // a store the compiler cannot prove dead, taken by no thread in practice
  if (s == T(-1.0)) sink[blockIdx.x] = s;
}

}  // namespace lagh

static lh_status probe(int32_t fp64, int32_t lanes, int64_t iters, void* sink, void* stream,
                       double* flops) {
  if (iters < 1 || iters > (int64_t(1) << 40) || !sink || lanes < 1 || lanes > 32) return LH_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return LH_ECUDA;
  const unsigned blocks = (unsigned)sms * 8u;  // 2048 resident threads per SM
  cudaStream_t s = (cudaStream_t)stream;
  if (fp64)
    lagh::fma_probe_kernel<double><<<blocks, 256, 0, s>>>((double*)sink, iters, 0.999999, 1e-7,
                                                          lanes);
  else
    lagh::fma_probe_kernel<float><<<blocks, 256, 0, s>>>((float*)sink, iters, 0.999999f, 1e-7f,
                                                         lanes);
  if (cudaGetLastError() != cudaSuccess) return LH_ECUDA;
  if (flops) *flops = 2.0 * 8.0 * (double)iters * blocks * 8.0 * lanes;
  return LH_OK;
}

extern "C" lh_status lh_peak_probe(int32_t fp64, int64_t iters, void* sink, void* stream,
                                   double* flops) {
  return probe(fp64, 32, iters, sink, stream, flops);
}

extern "C" lh_status lh_peak_probe_lanes(int32_t fp64, int32_t lanes, int64_t iters, void* sink,
                                         void* stream, double* flops) {
  return probe(fp64, lanes, iters, sink, stream, flops);
}
