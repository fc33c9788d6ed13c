// Batched kernels of the 2D shapes (see batch_kernels.cuh).
#include "batch_kernels.cuh"

namespace lagh {

template <int K, bool MIXED>
static bool pick(int ntt, BOps* out) {
  if (ntt == 256) { *out = make_batch_ops<2, K, MIXED, 256>(); return true; }
  if (ntt == 512) { *out = make_batch_ops<2, K, MIXED, 512>(); return true; }
  if (ntt == 1024) { *out = make_batch_ops<2, K, MIXED, 1024>(); return true; }
  return false;
}

bool get_batch_ops_2d(int k, bool mixed, int ntt, BOps* out) {
  if (k == 1) return mixed ? pick<1, true>(ntt, out) : pick<1, false>(ntt, out);
  if (k == 2) return mixed ? pick<2, true>(ntt, out) : pick<2, false>(ntt, out);
  if (k == 3) return mixed ? pick<3, true>(ntt, out) : pick<3, false>(ntt, out);
  return false;
}

}  // namespace lagh
