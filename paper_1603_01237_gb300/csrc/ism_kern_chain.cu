// The chains over sub-interval propagators (FP32 or FP64 tiles) and the intermediate states.
#include <mutex>
#include <set>
#include <utility>

#include "ism_launch_impl.cuh"

namespace ism {

template <typename R, int JC>
static cudaError_t chain_t(const ChainParams& p, size_t smem, cudaStream_t st) {
  dim3 grid(p.obj == 0 ? 2 : 1, p.B);
  const int threads = (chain_consumer_warps(p.d) + 1) * 32;   // consumer warps + one producer warp
  cudaError_t e = raise_smem_cap(reinterpret_cast<const void*>(k_chain<R, JC>));
  if (e != cudaSuccess) return e;
  k_chain<R, JC><<<grid, threads, smem, st>>>(p);
  return cudaGetLastError();
}

template <typename R>
static cudaError_t chain_d(const ChainParams& p, size_t smem, cudaStream_t st) {
  switch ((p.d + CHAIN_LANES - 1) / CHAIN_LANES) {   // columns per consumer thread
    case 1: return chain_t<R, 1>(p, smem, st);
    case 2: return chain_t<R, 2>(p, smem, st);
    case 3: return chain_t<R, 3>(p, smem, st);
    case 4: return chain_t<R, 4>(p, smem, st);
    case 5: return chain_t<R, 5>(p, smem, st);
    case 6: return chain_t<R, 6>(p, smem, st);
    case 7: return chain_t<R, 7>(p, smem, st);
    case 8: return chain_t<R, 8>(p, smem, st);
    default: return cudaErrorInvalidValue;
  }
}

template <typename R, int JC>
static cudaError_t fill_t(const ChainParams& p, cudaStream_t st) {
  using R2 = typename C2<R>::T;
  const size_t sm = (size_t)p.sblk * p.tile_stride * sizeof(R2);
  cudaError_t e = raise_smem_cap(reinterpret_cast<const void*>(k_fill<R, JC>));
  if (e != cudaSuccess) return e;
  k_fill<R, JC><<<dim3(p.Nc, p.B, 2), chain_consumer_warps(p.d) * 32, sm, st>>>(p);
  return cudaGetLastError();
}

template <typename R>
static cudaError_t fill_d(const ChainParams& p, cudaStream_t st) {
  switch ((p.d + CHAIN_LANES - 1) / CHAIN_LANES) {
    case 1: return fill_t<R, 1>(p, st);
    case 2: return fill_t<R, 2>(p, st);
    case 3: return fill_t<R, 3>(p, st);
    case 4: return fill_t<R, 4>(p, st);
    case 5: return fill_t<R, 5>(p, st);
    case 6: return fill_t<R, 6>(p, st);
    case 7: return fill_t<R, 7>(p, st);
    case 8: return fill_t<R, 8>(p, st);
    default: return cudaErrorInvalidValue;
  }
}

template <typename R>
static cudaError_t blockprod_t(const ChainParams& p, cudaStream_t st) {
  using R2 = typename C2<R>::T;
  const size_t sm = 3 * p.tile_stride * sizeof(R2);
  cudaError_t e = raise_smem_cap(reinterpret_cast<const void*>(k_blockprod<R>));
  if (e != cudaSuccess) return e;
  k_blockprod<R><<<dim3(p.Nc, p.B), 256, sm, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_chain(int prec, const ChainParams& p, size_t smem, cudaStream_t st) {
  cudaError_t e;
  if (p.Nc) {   // blocked: products of consecutive tiles first
    e = prec == 0 ? blockprod_t<double>(p, st) : blockprod_t<float>(p, st);
    if (e != cudaSuccess) return e;
  }
  e = prec == 0 ? chain_d<double>(p, smem, st) : chain_d<float>(p, smem, st);
  if (e != cudaSuccess) return e;
  if (p.Nc) {   // states inside the blocks
    e = prec == 0 ? fill_d<double>(p, st) : fill_d<float>(p, st);
    if (e != cudaSuccess) return e;
  }
  if (prec == 0) k_phi<double><<<dim3((p.N + 2 + 3) / 4, p.B), 128, 0, st>>>(p);
  else k_phi<float><<<dim3((p.N + 2 + 3) / 4, p.B), 128, 0, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_phi(int prec, const ChainParams& p, cudaStream_t st) {
  if (prec == 0) k_phi<double><<<dim3((p.N + 2 + 3) / 4, p.B), 128, 0, st>>>(p);
  else k_phi<float><<<dim3((p.N + 2 + 3) / 4, p.B), 128, 0, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_cheb_prep(int prec, const KParams& p, cudaStream_t st) {
  const long pairs = (long)p.B * p.N;
  if (pairs <= CHEB_WARP_PAIRS) {   // few pairs: one warp each, lowest latency
    if (prec == 0) k_cheb_prep_w<double><<<dim3(p.N, p.B), 32, 0, st>>>(p);
    else if (p.het) k_cheb_prep_w<float, true><<<dim3(p.N, p.B), 32, 0, st>>>(p);
    else k_cheb_prep_w<float><<<dim3(p.N, p.B), 32, 0, st>>>(p);
    return cudaGetLastError();
  }
  const unsigned grid = (unsigned)((pairs + CHEB_PAIRS - 1) / CHEB_PAIRS);
  if (prec == 0) k_cheb_prep<double><<<grid, 128, 0, st>>>(p);
  else if (p.het) k_cheb_prep<float, true><<<grid, 128, 0, st>>>(p);
  else k_cheb_prep<float><<<grid, 128, 0, st>>>(p);
  return cudaGetLastError();
}

size_t cheb_bytes(int prec) { return prec == 0 ? sizeof(Cheb<double>) : sizeof(Cheb<float>); }

cudaError_t raise_smem_cap(const void* kernel) {
  static std::mutex mu;
  static std::set<std::pair<const void*, int>> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  if (done.count({kernel, dev})) return cudaSuccess;
  int optin = 0;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  cudaFuncAttributes a;
  e = cudaFuncGetAttributes(&a, kernel);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)a.sharedSizeBytes);
  if (e == cudaSuccess) done.insert({kernel, dev});
  return e;
}

}  // namespace ism
