// ism_noalloc.cu -- ism_subinterval_grad_noalloc, the sub-interval gradient sweep for callers that
// cannot allocate device memory.
//
// Some callers cannot call cudaMalloc where they need this gradient: code running inside another
// framework's memory pool (the pool owns the device memory and a private cudaMalloc would bypass or
// fragment it), allocation-free real-time loops, and processes whose device-memory budget is fixed up
// front.  ism_plan allocates the sweep's scratch (the packed Hamiltonian, the partition, the per-step
// overlaps and the literal sub-problem's checkpoints) with cudaMalloc; this entry point keeps all of it
// in one file-scope __device__ array of ISM_NOALLOC_SCRATCH_BYTES instead and never calls cudaMalloc,
// cudaFree or any allocating library routine.  The caller passes device buffers for the inputs and outputs.
//
// The array is statically part of the module: every GPU that loads libism.so holds it until the
// process exits.  All calls share it, and it keeps the last call's contents; the only word that must
// start at zero (the status word) is cleared at the start of every call, everything else is written
// before it is read.  Two calls whose work overlaps on the GPU (different streams, or different host
// threads on one device) race on the array.
#include <cmath>
#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>

#include "ism.h"
#include "ism_kernels.cuh"
#include "ism_launch.h"

namespace {

constexpr size_t kScratchBytes = (size_t)ISM_NOALLOC_SCRATCH_BYTES;
__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// In host code `g_scratch` names a host-side stand-in, not a device address; the device address is
// looked up once per device with that device current and kept here.
constexpr int kMaxDevices = 128;
std::mutex g_mu;
unsigned char* g_scratch_dev[kMaxDevices] = {};

int scratch_for_current_device(unsigned char** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return ism::set_error(ISM_ECUDA, (std::string("cudaGetDevice: ") + cudaGetErrorString(e)).c_str());
  if (dev < 0 || dev >= kMaxDevices) return ism::set_error(ISM_EUNSUPPORTED, "device ordinal beyond the static scratch table");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_dev[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p)
      return ism::set_error(ISM_ECUDA, (std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e)).c_str());
    g_scratch_dev[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_dev[dev];
  return ISM_OK;
}

// Memory the kernels may dereference in place: device memory of the current GPU, or managed memory
// (another GPU's memory would be a peer access, or a fault without peer access enabled).
bool is_local_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  int dev = -1;
  return a.type == cudaMemoryTypeDevice && cudaGetDevice(&dev) == cudaSuccess && dev == a.device;
}

size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

extern "C" int ism_subinterval_grad_noalloc(const ism_problem* prob, int precision, const double* phi,
                                            const double* u, double* grad, double* Jn, void* cuda_stream) {
  if (!prob || !phi || !u || !grad) return ism::set_error(ISM_EINVAL, "null argument");
  const ism_problem& p = *prob;
  int rc = ism::validate_problem(p, precision);
  if (rc != ISM_OK) return rc;
  // the kernels below read a packed H0/H1 of the dense, tridiagonal or bit-flip layout: the grid kinds
  // (H0 = a few grid parameters, H1 unused) and the Pauli kind have other layouts and other sweeps
  if (p.kind != ISM_H_DENSE && p.kind != ISM_H_TRIDIAG && p.kind != ISM_H_BITFLIP)
    return ism::set_error(ISM_EUNSUPPORTED, "the allocation-free entry point covers the dense, tridiagonal and bit-flip kinds");
  if (!is_local_device_ptr(phi) || !is_local_device_ptr(u) || !is_local_device_ptr(grad) ||
      (Jn && !is_local_device_ptr(Jn)))
    return ism::set_error(ISM_EINVAL, "phi, u, grad and Jn must be device memory of the current GPU for the "
                                      "allocation-free entry point");
  // the kernel variant ism_plan picks for this problem (a tridiagonal H1 without a diagonal has its own)
  bool h1diag = true;
  if (p.kind == ISM_H_TRIDIAG) {
    h1diag = false;
    for (int e = 0; e < p.d; ++e) h1diag |= p.H1[e] != 0.0;
  }
  ism::KernelSet ks;
  if (!ism::select_kernels(precision, p.kind, p.d, &ks, h1diag, p.H0_imag || p.H1_imag))
    return ism::set_error(ISM_EUNSUPPORTED, "no compiled kernel for this kind and d");
  if (ks.large) return ism::set_error(ISM_EUNSUPPORTED, "the allocation-free entry point covers d <= 64");

  const int d = p.d, B = p.batch < 1 ? 1 : p.batch, GE = ks.G * ks.E;
  const size_t r1 = precision == ISM_FP64 ? sizeof(double) : sizeof(float);
  const size_t r2 = 2 * r1;
  std::vector<double> hd;
  std::vector<float> hf;
  size_t op_bytes;
  if (precision == ISM_FP64) {
    hd = ism::pack_op<double>(p.kind, d, p.H0, p.H1, ks.G, ks.E, p.H0_imag, p.H1_imag);
    op_bytes = hd.size() * r1;
  } else {
    hf = ism::pack_op<float>(p.kind, d, p.H0, p.H1, ks.G, ks.E, p.H0_imag, p.H1_imag);
    op_bytes = hf.size() * r1;
  }

  // the literal sub-problem's checkpoints: stride S ~ sqrt(longest sub-interval) (as ism_plan's default)
  const int nsmax = (p.Nt + p.N - 1) / p.N;
  int cks = (int)std::ceil(std::sqrt((double)nsmax));
  cks = cks < 1 ? 1 : (cks > nsmax ? nsmax : cks);
  const int nck = (nsmax + cks - 1) / cks;
  const size_t BN = (size_t)B * p.N;
  // scratch layout: op data | FP64 diag(H0) | j_n | beta_n | alpha | status | propagator parameters |
  // Bessel table | segment phases | FP32 controls | per-step overlaps | checkpoints | segment buffer
  const size_t off_h0d = up256(op_bytes);
  const size_t off_jn = off_h0d + up256(sizeof(double) * d);
  const size_t off_beta = off_jn + up256(sizeof(int) * (p.N + 1));
  const size_t off_alpha = off_beta + up256(sizeof(double) * p.N);
  const size_t off_status = off_alpha + up256(p.alpha ? sizeof(double) * p.Nt : 0);
  const size_t off_cheb = off_status + 256;
  const size_t off_ctab = off_cheb + up256((size_t)B * p.N * ism::cheb_bytes(precision));
  const size_t off_phase = off_ctab + up256(sizeof(double) * ism::BESSEL_TABLE);
  const size_t off_uf = off_phase + up256(sizeof(double2) * p.N);
  const size_t off_zs = off_uf + up256(sizeof(float) * (size_t)B * p.Nt);
  const size_t off_ckpt = off_zs + up256((size_t)B * ((size_t)p.Nt + p.N) * r2);
  const size_t off_segb = off_ckpt + up256(BN * nck * (precision == ISM_FP64 ? 1 : 2) * GE * r2);
  const size_t need = off_segb + up256(BN * cks * GE * r2);
  if (need > kScratchBytes) {
    std::string m = "problem needs " + std::to_string(need) + " bytes of scratch; the static scratch of the "
                    "allocation-free entry point holds " + std::to_string(kScratchBytes) + " bytes";
    return ism::set_error(ISM_EINVAL, m.c_str());
  }
  unsigned char* base = nullptr;
  if ((rc = scratch_for_current_device(&base)) != ISM_OK) return rc;

  const double tau = p.T / p.Nt;
  ism::Bounds bd = ism::bounds_of(p.kind, d, p.H0, p.H1, p.H0_imag, p.H1_imag);
  const double c0 = 0.5 * (bd.lo + bd.hi);
  std::vector<int> jn;
  std::vector<double> beta;
  std::vector<double2> phase;
  ism::partition(p.T, p.Nt, p.N, c0, &jn, &beta, &phase);

  cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
  cudaError_t e = cudaSuccess;
  auto h2d = [&](size_t off, const void* src, size_t n) {
    if (e == cudaSuccess && n) e = cudaMemcpyAsync(base + off, src, n, cudaMemcpyHostToDevice, st);
  };
  h2d(0, precision == ISM_FP64 ? (const void*)hd.data() : (const void*)hf.data(), op_bytes);
  std::vector<double> h0d(d);
  for (int e = 0; e < d; ++e) h0d[e] = p.kind == ISM_H_DENSE ? p.H0[(size_t)e * d + e] : p.H0[e];
  h2d(off_h0d, h0d.data(), sizeof(double) * d);
  h2d(off_jn, jn.data(), sizeof(int) * jn.size());
  h2d(off_beta, beta.data(), sizeof(double) * beta.size());
  if (p.alpha) h2d(off_alpha, p.alpha, sizeof(double) * p.Nt);
  std::vector<double> tab(ism::BESSEL_TABLE);
  ism::bessel_table(tab.data());
  h2d(off_ctab, tab.data(), sizeof(double) * tab.size());
  h2d(off_phase, phase.data(), sizeof(double2) * phase.size());
  if (e == cudaSuccess) e = cudaMemsetAsync(base + off_status, 0, sizeof(int), st);
  if (e != cudaSuccess) return ism::set_error(ISM_ECUDA, (std::string("scratch upload: ") + cudaGetErrorString(e)).c_str());

  ism::KParams k{};
  k.d = d; k.Nt = p.Nt; k.N = p.N; k.B = B; k.ldm = d | 1; k.dpad = d; k.tile_stride = 0;
  k.tau = tau; k.T = p.T; k.c0 = 0.5 * (bd.lo + bd.hi); k.r0 = 0.5 * (bd.hi - bd.lo); k.h1n = bd.h1;
  k.tol = precision == ISM_FP64 ? 1e-17 : 1e-10;
  k.rho = 0.0; k.w = p.objective == ISM_OBJ_OVERLAP ? 1.0 : 2.0;
  k.jn = reinterpret_cast<const int*>(base + off_jn);
  k.beta = reinterpret_cast<const double*>(base + off_beta);
  k.alpha = p.alpha ? reinterpret_cast<const double*>(base + off_alpha) : nullptr;
  k.H = base;
  k.H0d = reinterpret_cast<const double*>(base + off_h0d);
  k.u = const_cast<double*>(u);
  k.phi = reinterpret_cast<const double2*>(phi);
  k.M = nullptr;
  k.traj = nullptr;
  k.traj2 = nullptr;
  k.zs = base + off_zs;
  k.ckpt = base + off_ckpt;
  k.segb = base + off_segb;
  k.cks = cks;
  k.nck = nck;
  k.grad = grad;
  k.Jn = Jn;
  k.err = nullptr;
  k.status = reinterpret_cast<int*>(base + off_status);
  k.count = nullptr;
  k.psin = nullptr;
  k.chin = nullptr;
  k.form = 0;
  k.update = 0;
  k.max_spin = 1 << 22;
  k.cheb = base + off_cheb;
  k.pen = nullptr;
  k.uf = reinterpret_cast<float*>(base + off_uf);
  k.phase = reinterpret_cast<const double2*>(base + off_phase);
  k.ctab = reinterpret_cast<const double*>(base + off_ctab);
  // non-finite controls or states: ISM_ENONFINITE (the propagator bound below would drop a NaN)
  {
    const long nu = (long)B * p.Nt, nphi = 2L * B * (p.N + 1) * d;
    ism::k_check_finite<<<(unsigned)std::min<long>(1024, (nu + 255) / 256), 256, 0, st>>>(u, nu, k.status);
    ism::k_check_finite<<<(unsigned)std::min<long>(1024, (nphi + 255) / 256), 256, 0, st>>>(phi, nphi, k.status);
    if ((e = cudaGetLastError()) != cudaSuccess)
      return ism::set_error(ISM_ECUDA, (std::string("launch: ") + cudaGetErrorString(e)).c_str());
  }
  if ((e = ism::launch_cheb_prep(precision, k, st)) != cudaSuccess)
    return ism::set_error(ISM_ECUDA, (std::string("launch: ") + cudaGetErrorString(e)).c_str());
  if ((e = ks.subinterval(k, st)) != cudaSuccess)
    return ism::set_error(ISM_ECUDA, (std::string("launch: ") + cudaGetErrorString(e)).c_str());
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess)
    return ism::set_error(ISM_ECUDA, (std::string("stream: ") + cudaGetErrorString(e)).c_str());
  int status = 0;
  if ((e = cudaMemcpy(&status, base + off_status, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return ism::set_error(ISM_ECUDA, (std::string("status read: ") + cudaGetErrorString(e)).c_str());
  if (status & ism::ST_TIMEOUT) return ism::set_error(ISM_ETIMEOUT, "a bounded device-side wait gave up");
  if (status & ism::ST_KOVERFLOW) return ism::set_error(ISM_EUNSUPPORTED, "Chebyshev series needed more terms than compiled");
  if (status & ism::ST_NONFINITE) return ism::set_error(ISM_ENONFINITE, "non-finite value in a control or a result");
  if (status & ism::ST_SPECTRUM)
    return ism::set_error(ISM_EUNSUPPORTED, "controls so large that a time step needs more Chebyshev sub-steps than the limit");
  ism::clear_error();
  return ISM_OK;
}
