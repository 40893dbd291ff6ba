// ism_launch_impl.cuh -- launcher templates shared by the per-structure translation units.
#pragma once
#include "ism_kernels.cuh"
#include "ism_launch.h"

namespace ism {

template <typename R, class Op>
size_t op_smem_bytes() {
  return (size_t)Op::SMEM_WORDS * sizeof(R);
}

template <typename R, class Op>
cudaError_t launch_assemble_t(const KParams& p, cudaStream_t st) {
  constexpr int GPB = 128 / Op::G;
  const long groups = (long)p.B * p.N * p.dpad;
  const long grid = (groups + GPB - 1) / GPB;
  const size_t smem = op_smem_bytes<R, Op>();
  if (smem > 40 * 1024) {   // leave room for the static shared memory under the 48 KB default
    cudaError_t e = raise_smem_cap(reinterpret_cast<const void*>(k_assemble<R, Op>));
    if (e != cudaSuccess) return e;
  }
  k_assemble<R, Op><<<(unsigned)grid, 128, smem, st>>>(p);
  return cudaGetLastError();
}

// The sub-problems of Algorithm 1 step (c): p.form = 1 (two-trajectory form of a first local step)
// runs k_subfwd, p.form = 0 (literal sub-problem from phi) the checkpointed k_subinterval.
template <typename R, class Op>
cudaError_t launch_subinterval_t(const KParams& p, cudaStream_t st) {
  constexpr int GPB = 128 / Op::G;
  const long groups = (long)p.B * p.N;
  const long grid = (groups + GPB - 1) / GPB;
  const size_t smem = op_smem_bytes<R, Op>();
  const void* fn = p.form ? reinterpret_cast<const void*>(k_subfwd<R, Op>) : reinterpret_cast<const void*>(k_subinterval<R, Op>);
  if (smem > 40 * 1024) {
    cudaError_t e = raise_smem_cap(fn);
    if (e != cudaSuccess) return e;
  }
  if constexpr (sizeof(R) == 4 && !Op::CN && Op::DP_SMEM == 0) {   // heterogeneous batches: FP32 structured kinds
    if (p.het) {
      k_subfwd<R, Op, true><<<(unsigned)grid, 128, smem, st>>>(p);
      return cudaGetLastError();
    }
  }
  if (p.form) k_subfwd<R, Op><<<(unsigned)grid, 128, smem, st>>>(p);
  else k_subinterval<R, Op><<<(unsigned)grid, 128, smem, st>>>(p);
  return cudaGetLastError();
}

template <typename R, class Op>
cudaError_t launch_sweeps2_t(const KParams& p, cudaStream_t st) {
  constexpr int GPB = 128 / Op::G;
  const long groups = (long)p.B * p.N;
  const long grid = (groups + GPB - 1) / GPB;
  const size_t smem = op_smem_bytes<R, Op>();
  if (smem > 40 * 1024) {
    cudaError_t e = raise_smem_cap(reinterpret_cast<const void*>(k_sweeps2<R, Op>));
    if (e != cudaSuccess) return e;
  }
  k_sweeps2<R, Op><<<dim3((unsigned)grid, 2), 128, smem, st>>>(p);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_gradpass<R><<<dim3(p.N, p.B), 256, 0, st>>>(p, Op::G * Op::E);
  return cudaGetLastError();
}

template <typename R, class Op>
cudaError_t launch_gsweep_t(const KParams& p, cudaStream_t st) {
  constexpr int GPB = 128 / Op::G;
  const long grid = ((long)p.B + GPB - 1) / GPB;
  const size_t smem = op_smem_bytes<R, Op>();
  if (smem > 40 * 1024) {
    cudaError_t e = raise_smem_cap(reinterpret_cast<const void*>(k_gsweep<R, Op>));
    if (e != cudaSuccess) return e;
  }
  if constexpr (sizeof(R) == 4 && !Op::CN && Op::DP_SMEM == 0) {
    if (p.het) {
      k_gsweep<R, Op, true><<<dim3((unsigned)grid, p.obj == 0 ? 2 : 1), 128, smem, st>>>(p);
      return cudaGetLastError();
    }
  }
  k_gsweep<R, Op><<<dim3((unsigned)grid, p.obj == 0 ? 2 : 1), 128, smem, st>>>(p);
  return cudaGetLastError();
}

// OpA: lane layout of the throughput-bound assembly (few lanes, many elements per lane);
// OpS: lane layout of the latency-bound sub-interval sweep (more lanes per state).
// SWEEPS2: also build the concurrent two-trajectory sweeps (otherwise the sub-problems of the
// two-trajectory form run in k_subinterval).
template <typename R, class OpA, class OpS = OpA, bool SWEEPS2 = true>
void fill_set(KernelSet* ks) {
  ks->assemble = &launch_assemble_t<R, OpA>;
  ks->subinterval = &launch_subinterval_t<R, OpS>;
  if constexpr (SWEEPS2) ks->sweeps2 = &launch_sweeps2_t<R, OpS>;
  else ks->sweeps2 = nullptr;
  ks->gsweep = &launch_gsweep_t<R, OpS>;
  if constexpr (sizeof(R) == 4 && OpA::PACKED && OpA::G != OpS::G) ks->gsweep_wide = &launch_gsweep_t<R, OpA>;
  else ks->gsweep_wide = nullptr;
  ks->GW = OpA::G;
  ks->G = OpS::G;
  ks->E = OpS::E;
  ks->GA = OpA::G;
  ks->op_smem = op_smem_bytes<R, OpS>();
}

}  // namespace ism
