// The chains over sub-interval propagators (FP32 or FP64 tiles) and the intermediate states.
#include "ism_launch_impl.cuh"

namespace ism {

cudaError_t launch_chain(int prec, const ChainParams& p, size_t smem, cudaStream_t st) {
  dim3 grid(p.obj == 0 ? 2 : 1, p.B);
  cudaError_t e;
  if (prec == 0) {
    e = cudaFuncSetAttribute(k_chain<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_chain<double><<<grid, 256, smem, st>>>(p);
  } else {
    e = cudaFuncSetAttribute(k_chain<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_chain<float><<<grid, 256, smem, st>>>(p);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_phi<0><<<p.B, 1024, 0, st>>>(p);
  return cudaGetLastError();
}

}  // namespace ism
