// Tridiagonal Hamiltonians with the Crank-Nicolson time step of Sec. 3 (FP64, d <= 64): the
// lane layouts of the Chebyshev build; the sub-problems always run the one-group sweep (k_subinterval).
#include "ism_launch_impl.cuh"

namespace ism {

template <bool HB>
static bool pick_cn(int d, KernelSet* ks) {
  using R = double;
  const int E = (d + 15) / 16;
  switch (E) {
    case 1: fill_set<R, OpTridiagCN<R, 8, 2, HB>, OpTridiagCN<R, 16, 1, HB>, false>(ks); return true;
    case 2: fill_set<R, OpTridiagCN<R, 8, 4, HB>, OpTridiagCN<R, 16, 2, HB>, false>(ks); return true;
    case 3: fill_set<R, OpTridiagCN<R, 8, 6, HB>, OpTridiagCN<R, 16, 3, HB>, false>(ks); return true;
    case 4: fill_set<R, OpTridiagCN<R, 8, 8, HB>, OpTridiagCN<R, 16, 4, HB>, false>(ks); return true;
    default: return false;
  }
}

bool kernels_tridiag_cn(int prec, int d, bool h1diag, KernelSet* ks) {
  if (prec != 0 || d < 1 || d > 64) return false;
  return h1diag ? pick_cn<true>(d, ks) : pick_cn<false>(d, ks);
}

}  // namespace ism
