// Tridiagonal Hamiltonians (rigid rotor in the |j, m=0> basis): d <= 64, 16 lanes per state.
#include "ism_launch_impl.cuh"

namespace ism {

// assembly: 8 lanes x ceil(d/8) elements; sweep: 16 lanes x ceil(d/16) elements
template <typename R>
static bool pick(int d, KernelSet* ks) {
  const int E = (d + 15) / 16;
  switch (E) {
    case 1: fill_set<R, OpTridiag<R, 8, 2>, OpTridiag<R, 16, 1>>(ks); return true;
    case 2: fill_set<R, OpTridiag<R, 8, 4>, OpTridiag<R, 16, 2>>(ks); return true;
    case 3: fill_set<R, OpTridiag<R, 8, 6>, OpTridiag<R, 16, 3>>(ks); return true;
    case 4: fill_set<R, OpTridiag<R, 8, 8>, OpTridiag<R, 16, 4>>(ks); return true;
    default: return false;
  }
}

bool kernels_tridiag(int prec, int d, KernelSet* ks) {
  if (d < 1 || d > 64) return false;
  return prec == 0 ? pick<double>(d, ks) : pick<float>(d, ks);
}

}  // namespace ism
