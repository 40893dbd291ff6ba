// Tridiagonal Hamiltonians (rigid rotor in the |j, m=0> basis): d <= 64, 16 lanes per state.
#include "ism_launch_impl.cuh"

namespace ism {

// assembly: 8 lanes x ceil(d/8) elements; sweep: 16 lanes x ceil(d/16) elements.  HB: H1 has a diagonal.
template <typename R, bool HB>
static bool pick(int d, KernelSet* ks) {
  const int E = (d + 15) / 16;
  switch (E) {
    case 1: fill_set<R, OpTridiag<R, 8, 2, HB>, OpTridiag<R, 16, 1, HB>>(ks); return true;
    case 2: fill_set<R, OpTridiag<R, 8, 4, HB>, OpTridiag<R, 16, 2, HB>>(ks); return true;
    case 3: fill_set<R, OpTridiag<R, 8, 6, HB>, OpTridiag<R, 16, 3, HB>>(ks); return true;
    case 4: fill_set<R, OpTridiag<R, 8, 8, HB>, OpTridiag<R, 16, 4, HB>>(ks); return true;
    default: return false;
  }
}

bool kernels_tridiag(int prec, int d, bool h1diag, KernelSet* ks) {
  if (d < 1 || d > 64) return false;
  if (h1diag) return prec == 0 ? pick<double, true>(d, ks) : pick<float, true>(d, ks);
  return prec == 0 ? pick<double, false>(d, ks) : pick<float, false>(d, ks);
}

}  // namespace ism
