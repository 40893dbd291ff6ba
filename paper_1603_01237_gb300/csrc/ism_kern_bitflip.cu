// Diagonal H0 plus bit-flip H1 = sum_i h_i X_i (spin systems): d = 2^q, 2 <= d <= 64.
#include "ism_launch_impl.cuh"

namespace ism {

template <typename R>
static bool pick(int d, KernelSet* ks) {
  switch (d) {
    case 2: fill_set<R, OpBitflip<R, 2, 1>>(ks); return true;
    case 4: fill_set<R, OpBitflip<R, 4, 1>>(ks); return true;
    case 8: fill_set<R, OpBitflip<R, 4, 2>, OpBitflip<R, 8, 1>>(ks); return true;
    case 16: fill_set<R, OpBitflip<R, 4, 4>, OpBitflip<R, 16, 1>>(ks); return true;
    case 32: fill_set<R, OpBitflip<R, 8, 4>, OpBitflip<R, 16, 2>>(ks); return true;
    case 64: fill_set<R, OpBitflip<R, 8, 8>, OpBitflip<R, 16, 4>>(ks); return true;
    default: return false;
  }
}

bool kernels_bitflip(int prec, int d, KernelSet* ks) {
  return prec == 0 ? pick<double>(d, ks) : pick<float>(d, ks);
}

}  // namespace ism
