// The chains over sub-interval propagators (FP32 or FP64 tiles) and the intermediate states.
#include "ism_launch_impl.cuh"

namespace ism {

cudaError_t launch_chain(int prec, const ChainParams& p, size_t smem, cudaStream_t st) {
  dim3 grid(p.obj == 0 ? 2 : 1, p.B);
  const int threads = (chain_consumer_warps(p.d) + 1) * 32;   // consumer warps + one producer warp
  cudaError_t e;
  if (prec == 0) {
    e = cudaFuncSetAttribute(k_chain<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_chain<double><<<grid, threads, smem, st>>>(p);
  } else {
    e = cudaFuncSetAttribute(k_chain<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_chain<float><<<grid, threads, smem, st>>>(p);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (prec == 0) k_phi<double><<<dim3(p.N + 2, p.B), 128, 0, st>>>(p);
  else k_phi<float><<<dim3(p.N + 2, p.B), 128, 0, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_cheb_prep(int prec, const KParams& p, cudaStream_t st) {
  if (prec == 0) k_cheb_prep<double><<<dim3(p.N, p.B), 32, 0, st>>>(p);
  else k_cheb_prep<float><<<dim3(p.N, p.B), 32, 0, st>>>(p);
  return cudaGetLastError();
}

size_t cheb_bytes(int prec) { return prec == 0 ? sizeof(Cheb<double>) : sizeof(Cheb<float>); }

}  // namespace ism
