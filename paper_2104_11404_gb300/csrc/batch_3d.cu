// Batched kernels of the 3D shapes (see batch_kernels.cuh).
#include "batch_kernels.cuh"

namespace lagh {

template <int K, bool MIXED>
static bool pick(int ntt, int qpt, BOps* out) {
  if (qpt != 1) return false;
  if (ntt == 256) { *out = make_batch_ops<3, K, MIXED, 256, 1>(); return true; }
  if (ntt == 512) { *out = make_batch_ops<3, K, MIXED, 512, 1>(); return true; }
  return false;
}

bool get_batch_ops_3d(int k, bool mixed, int ntt, int qpt, BOps* out) {
  if (k == 1) return mixed ? pick<1, true>(ntt, qpt, out) : pick<1, false>(ntt, qpt, out);
  if (k == 2) return mixed ? pick<2, true>(ntt, qpt, out) : pick<2, false>(ntt, qpt, out);
  return false;
}

}  // namespace lagh
