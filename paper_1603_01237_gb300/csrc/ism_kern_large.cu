// Spin chains of 7 to 10 sites (d = 128 .. 1024): diagonal H0, bit-flip H1, one state per CTA.
#include "ism_large.cuh"
#include "ism_launch.h"

namespace ism {

template <typename R, class Op>
cudaError_t launch_lsweep_t(const KParams& p, cudaStream_t st) {
  if constexpr (sizeof(R) == 4) {   // heterogeneous batches (mixed precision only)
    if (p.het) {
      k_lsweep<R, Op, true><<<dim3(p.obj == 0 ? 2 : 1, p.B), Op::NT, 0, st>>>(p);
      return cudaGetLastError();
    }
  }
  k_lsweep<R, Op><<<dim3(p.obj == 0 ? 2 : 1, p.B), Op::NT, 0, st>>>(p);
  return cudaGetLastError();
}

template <typename R, class Op>
cudaError_t launch_lsub_t(const KParams& p, cudaStream_t st) {
  if constexpr (sizeof(R) == 4) {
    if (p.het) {
      k_lsub<R, Op, true><<<dim3(p.N, p.B), Op::NT, 0, st>>>(p);
      return cudaGetLastError();
    }
  }
  k_lsub<R, Op><<<dim3(p.N, p.B), Op::NT, 0, st>>>(p);
  return cudaGetLastError();
}

// Sweep layout (WS warps x ES elements per thread) and sub-interval layout (W warps x 4 elements)
// are chosen separately: the sweep is one CTA per SM on a sequential chain, the sub-interval kernel
// N CTAs sharing the GPU.
template <typename R, int WS, int ES, int W>
static void fill_large(KernelSet* ks) {
  using OpS = OpBitflipCTA<R, WS, ES>;
  using Op = OpBitflipCTA<R, W, 4>;
  static_assert(OpS::D == Op::D, "both layouts cover the same dimension");
  ks->large = true;
  ks->lsweep = &launch_lsweep_t<R, OpS>;
  ks->subinterval = &launch_lsub_t<R, Op>;
  ks->G = Op::NT;
  ks->E = Op::E;
  ks->W = W;
}

// Measured at d = 1024 (FP32): 4 elements per thread over 8 warps, ~640 ns per application of H;
// 16 elements over 2 warps, 2.2x slower (two of four SM sub-partitions idle, longer per-thread
// chains).  The exchanges, not the arithmetic, set the pace, so both kernels use the 4-element layout.
template <typename R>
static bool pick(int d, KernelSet* ks) {
  switch (d) {
    case 128: fill_large<R, 1, 4, 1>(ks); return true;
    case 256: fill_large<R, 2, 4, 2>(ks); return true;
    case 512: fill_large<R, 4, 4, 4>(ks); return true;
    case 1024: fill_large<R, 8, 4, 8>(ks); return true;
    default: return false;
  }
}

bool kernels_large_bitflip(int prec, int d, KernelSet* ks) {
  return prec == 0 ? pick<double>(d, ks) : pick<float>(d, ks);
}

}  // namespace ism
