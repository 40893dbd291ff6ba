// The sequential chain over sub-interval propagators (FP32 or FP64 tiles), one CTA per problem.
#include "ism_launch_impl.cuh"

namespace ism {

cudaError_t launch_chain(int prec, const ChainParams& p, size_t smem, cudaStream_t st) {
  cudaError_t e;
  if (prec == 0) {
    e = cudaFuncSetAttribute(k_chain<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_chain<double><<<p.B, 256, smem, st>>>(p);
  } else {
    e = cudaFuncSetAttribute(k_chain<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_chain<float><<<p.B, 256, smem, st>>>(p);
  }
  return cudaGetLastError();
}

}  // namespace ism
