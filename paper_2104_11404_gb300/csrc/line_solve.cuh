// Banded Cholesky substitution along one node line, shared by the exact
// tensor-product preconditioner of the context CG (cg.cu) and the in-CTA CG of
// the batched form (batch_kernels.cuh).
#pragma once

#include <stdint.h>

namespace lagh {

// Forward and backward substitution along one node line of w (m entries,
// stride apart): w <- (L L^T)^-1 w with the banded Cholesky factor L of the
// assembled 1D matrix.  Row i of the table F holds d_i = 1 / L_ii, the scaled
// forward coefficients d_i L_{i,i-q} and the scaled backward coefficients
// d_i L_{i+q,i} (q = 1..K), so each substitution step has one dependent FMA.
template <int K>
__device__ __forceinline__ void line_solve(double* L, int64_t stride, int m,
                                           const double* __restrict__ F) {
  constexpr int W = 2 * K + 1;
  double win[K];
#pragma unroll
  for (int q = 0; q < K; ++q) win[q] = 0.0;
  double b = m > 0 ? L[0] : 0.0;
  for (int i = 0; i < m; ++i) {  // y_i = d_i b_i - sum_q d_i L_{i,i-q} y_{i-q}
    const double* Fi = F + (int64_t)i * W;
    const double bn = (i + 1 < m) ? L[(i + 1) * stride] : 0.0;  // next input, off the chain
    double s = Fi[0] * b;
#pragma unroll
    for (int q = K; q >= 1; --q) s = fma(-Fi[q], win[q - 1], s);
#pragma unroll
    for (int q = K - 1; q > 0; --q) win[q] = win[q - 1];
    win[0] = s;
    L[i * stride] = s;
    b = bn;
  }
#pragma unroll
  for (int q = 0; q < K; ++q) win[q] = 0.0;
  double y = m > 0 ? L[(m - 1) * stride] : 0.0;
  for (int i = m - 1; i >= 0; --i) {  // x_i = d_i y_i - sum_q d_i L_{i+q,i} x_{i+q}
    const double* Fi = F + (int64_t)i * W;
    const double yn = i > 0 ? L[(i - 1) * stride] : 0.0;
    double s = Fi[0] * y;
#pragma unroll
    for (int q = K; q >= 1; --q) s = fma(-Fi[K + q], win[q - 1], s);
#pragma unroll
    for (int q = K - 1; q > 0; --q) win[q] = win[q - 1];
    win[0] = s;
    L[i * stride] = s;
    y = yn;
  }
}

}  // namespace lagh
