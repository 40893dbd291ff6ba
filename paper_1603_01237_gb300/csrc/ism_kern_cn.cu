// The Crank-Nicolson time step of Sec. 3 (d <= 64) for the tridiagonal, bit-flip and dense kinds, in
// FP64 and in FP32 propagation (mixed mode: the Cayley step is unitary by construction, so its FP32
// rounding does not build up a norm or phase drift the way a truncated series would; states at the
// partition, overlaps and the update stay FP64): the lane layouts of the Chebyshev builds; the
// sub-problems always run the one-group sweep (k_subinterval).
#include "ism.h"
#include "ism_launch_impl.cuh"

namespace ism {

template <typename R, bool HB>
static bool pick_cn(int d, KernelSet* ks) {
  const int E = (d + 15) / 16;
  switch (E) {
    case 1: fill_set<R, OpTridiagCN<R, 8, 2, HB>, OpTridiagCN<R, 16, 1, HB>, false>(ks); return true;
    case 2: fill_set<R, OpTridiagCN<R, 8, 4, HB>, OpTridiagCN<R, 16, 2, HB>, false>(ks); return true;
    case 3: fill_set<R, OpTridiagCN<R, 8, 6, HB>, OpTridiagCN<R, 16, 3, HB>, false>(ks); return true;
    case 4: fill_set<R, OpTridiagCN<R, 8, 8, HB>, OpTridiagCN<R, 16, 4, HB>, false>(ks); return true;
    default: return false;
  }
}

template <typename R>
static bool pick_bitflip_cn(int d, KernelSet* ks) {
  switch (d) {
    case 2: fill_set<R, OpBitflipCN<R, 2, 1>, OpBitflipCN<R, 2, 1>, false>(ks); return true;
    case 4: fill_set<R, OpBitflipCN<R, 4, 1>, OpBitflipCN<R, 4, 1>, false>(ks); return true;
    case 8: fill_set<R, OpBitflipCN<R, 4, 2>, OpBitflipCN<R, 8, 1>, false>(ks); return true;
    case 16: fill_set<R, OpBitflipCN<R, 4, 4>, OpBitflipCN<R, 16, 1>, false>(ks); return true;
    case 32: fill_set<R, OpBitflipCN<R, 8, 4>, OpBitflipCN<R, 16, 2>, false>(ks); return true;
    case 64: fill_set<R, OpBitflipCN<R, 8, 8>, OpBitflipCN<R, 16, 4>, false>(ks); return true;
    default: return false;
  }
}

template <typename R>
static bool pick_dense_cn(int d, KernelSet* ks) {
  switch ((d + 15) / 16) {
    case 1: fill_set<R, OpDenseCN<R, 16, 1>, OpDenseCN<R, 16, 1>, false>(ks); return true;
    case 2: fill_set<R, OpDenseCN<R, 16, 2>, OpDenseCN<R, 16, 2>, false>(ks); return true;
    case 3: fill_set<R, OpDenseCN<R, 16, 3>, OpDenseCN<R, 16, 3>, false>(ks); return true;
    case 4: fill_set<R, OpDenseCN<R, 16, 4>, OpDenseCN<R, 16, 4>, false>(ks); return true;
    default: return false;
  }
}

template <typename R>
static bool pick_kind(int kind, int d, bool h1diag, KernelSet* ks) {
  switch (kind) {
    case ISM_H_TRIDIAG: return h1diag ? pick_cn<R, true>(d, ks) : pick_cn<R, false>(d, ks);
    case ISM_H_BITFLIP: return pick_bitflip_cn<R>(d, ks);
    case ISM_H_DENSE: return pick_dense_cn<R>(d, ks);
    default: return false;
  }
}

bool kernels_cn(int prec, int kind, int d, bool h1diag, KernelSet* ks) {
  if (d < 1 || d > 64) return false;
  return prec == 0 ? pick_kind<double>(kind, d, h1diag, ks) : pick_kind<float>(kind, d, h1diag, ks);
}

}  // namespace ism
