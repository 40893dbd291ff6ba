// Dense complex Hermitian H0, H1 (generic problems): d <= 64, 16 lanes per state, the real and
// imaginary parts of H staged in shared memory.
#include "ism_launch_impl.cuh"

namespace ism {

template <typename R>
static bool pick(int d, KernelSet* ks) {
  const int E = (d + 15) / 16;
  switch (E) {
    case 1: fill_set<R, OpDense<R, 16, 1, true>>(ks); return true;
    case 2: fill_set<R, OpDense<R, 16, 2, true>>(ks); return true;
    case 3: fill_set<R, OpDense<R, 16, 3, true>>(ks); return true;
    case 4: fill_set<R, OpDense<R, 16, 4, true>>(ks); return true;
    default: return false;
  }
}

bool kernels_dense_cx(int prec, int d, KernelSet* ks) {
  if (d < 1 || d > 64) return false;
  return prec == 0 ? pick<double>(d, ks) : pick<float>(d, ks);
}

}  // namespace ism
