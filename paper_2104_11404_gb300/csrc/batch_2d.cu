// Batched kernels of the 2D shapes, one point per thread (see batch_kernels.cuh).
#include "batch_kernels.cuh"

namespace lagh {

template <int K, bool MIXED>
static bool pick(int ntt, int qpt, BOps* out) {
  if (qpt != 1) return false;
  if (ntt == 256) { *out = make_batch_ops<2, K, MIXED, 256, 1>(); return true; }
  if (ntt == 512) { *out = make_batch_ops<2, K, MIXED, 512, 1>(); return true; }
  if (ntt == 1024) { *out = make_batch_ops<2, K, MIXED, 1024, 1>(); return true; }
  return false;
}

bool get_batch_ops_2d_q1(int k, bool mixed, int ntt, int qpt, BOps* out) {
  if (k == 1) return mixed ? pick<1, true>(ntt, qpt, out) : pick<1, false>(ntt, qpt, out);
  if (k == 2) return mixed ? pick<2, true>(ntt, qpt, out) : pick<2, false>(ntt, qpt, out);
  if (k == 3) return mixed ? pick<3, true>(ntt, qpt, out) : pick<3, false>(ntt, qpt, out);
  return false;
}

}  // namespace lagh
