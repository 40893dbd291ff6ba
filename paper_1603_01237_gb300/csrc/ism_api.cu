// ism_api.cu -- the C ABI declared in include/ism.h: plan creation and validation, the partition
// and weights of Sec. 2, spectral bounds for the Chebyshev propagator, and the orchestration of the
// hot-path kernels on the plan's stream.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <initializer_list>
#include <string>
#include <vector>

#include "ism.h"
#include "ism_kernels.cuh"
#include "ism_launch.h"
#include "ism_gp.h"
#include "ism_tc.h"

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

}  // namespace

namespace ism {
int set_error(int code, const char* msg) { return fail(code, msg); }
void clear_error() { g_err.clear(); }

void partition(double T, int Nt, int N, double c0, std::vector<int>* jn, std::vector<double>* beta,
               std::vector<double2>* phase) {
  const double tau = T / Nt;
  jn->assign(N + 1, 0);
  for (int n = 0; n <= N; ++n) (*jn)[n] = (int)(((long long)n * Nt) / N);
  if (beta) {
    beta->assign(N, 0.0);
    for (int n = 0; n < N; ++n) (*beta)[n] = T / ((*jn)[n + 1] * tau - (*jn)[n] * tau);
  }
  if (phase) {
    phase->assign(N, make_double2(1.0, 0.0));
    for (int n = 0; n < N; ++n) {
      const double ph = c0 * tau * (double)((*jn)[n + 1] - (*jn)[n]);
      (*phase)[n] = make_double2(std::cos(ph), std::sin(ph));
    }
  }
}
}  // namespace ism

namespace {

#define ISM_CUDA_TRY(expr)                                                                    \
  do {                                                                                        \
    cudaError_t e_ = (expr);                                                                  \
    if (e_ != cudaSuccess) return fail(ISM_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
  } while (0)

bool all_finite(const double* x, long n) {
  for (long i = 0; i < n; ++i)
    if (!std::isfinite(x[i])) return false;
  return true;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// ISM_EINVAL when an argument is device memory of another GPU than the plan's: the kernels use device
// arrays in place, and another GPU's memory would be a peer access (or a fault without peer access).
int check_device_args(int dev, std::initializer_list<const void*> ptrs) {
  for (const void* p : ptrs) {
    if (!p) continue;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    if (a.type == cudaMemoryTypeDevice && a.device != dev)
      return fail(ISM_EINVAL, "an array argument is device memory of GPU " + std::to_string(a.device) +
                                  ", not of the plan's GPU " + std::to_string(dev));
  }
  return ISM_OK;
}

// err_hist[b][k] = sum_n err[b][n]  (Algorithm 1 (e)), one warp per problem
__global__ void k_err_sum(const double* err, int N, int B, double* hist, int stride, int k) {
  const int b = blockIdx.x;
  double s = 0.0;
  for (int n = threadIdx.x; n < N; n += 32) s += err[(long)b * N + n];
  for (int m = 16; m >= 1; m >>= 1) s += __shfl_xor_sync(0xffffffffu, s, m);
  if (threadIdx.x == 0) hist[(long)b * stride + k] = s;
}

}  // namespace

struct ism_plan_s {
  int d = 0, kind = 0, obj = 0, Nt = 0, N = 0, B = 1, prec = 0, L = 1;
  double T = 0, tau = 0, rho = 0, tol = 0, w = 1;
  int max_spin = 0;
  int form = 1;   // sub-problem form in ism_iterate: 1 literal, 2 Theorem 2 (first local step)
  int scheme = ISM_SCHEME_CHEBYSHEV;
  bool gp = false;                       // grid (Gross-Pitaevskii) kind
  double gpL = 0, gpxmin = 0, gpg = 0;   // its grid length, origin and nonlinearity
  int gppot = 0;                         // potential: 0 harmonic (x - u)^2/2, 1 double well
  int m = 1, q = 0;                      // controls per step; bits of d (Pauli kind)
  bool pauli = false;
  bool wide = false;                     // direct sweeps in the wide lane layout
  double nrm_psi_i = 0, nrm_psi_f = 0;   // |psi_i|^2, |psi_f|^2 (references of the renormalisation)
  double* dnrm = nullptr;                // [B][N+1][2] squared norms of psi(t_n), chi(t_n) (direct sweeps)
  double* dwts = nullptr;                // Pauli kind: [m][q][2] control weights
  void* dcxy = nullptr;                  // Pauli kind: [B][Nt][2q] step coefficients (R)
  double gpdw = 0;                       // double-well separation D
  double c0 = 0, r0 = 0, h1n = 0;
  ism::KernelSet ks;
  int ldm = 0, dpad = 0;
  long tst = 0;
  size_t r2 = 0;  // bytes of one complex element of the propagation precision
  cudaStream_t st = nullptr;
  int dev = 0;
  void* dH = nullptr;
  double* dH0d = nullptr;   // FP64 diagonal of H0
  int* djn = nullptr;
  double* dbeta = nullptr;
  double2* dab = nullptr;   // (a_n, b_n), n = 0..N
  double2* dphase = nullptr;   // (cos, sin) of c0 tau (steps of sub-interval n)
  unsigned char* dcheb = nullptr;   // propagator parameters per (problem, n)
  unsigned char* dstage = nullptr;  // chain results before FP64 conversion
  double* dpen = nullptr;           // penalty sums per (problem, n)
  double* dctab = nullptr;          // Bessel series table
  double* dalpha = nullptr;
  double* dO = nullptr;
  double2* dpsi_i = nullptr;
  double2* dpsi_f = nullptr;
  void* dM = nullptr;
  double2* dpsin = nullptr;
  double2* dchin = nullptr;
  double2* dphi = nullptr;
  void* dtraj = nullptr;
  void* dgptab = nullptr;           // grid kinds: twiddle, kinetic-factor and grid tables
  void* dtraj2 = nullptr;
  bool use_sw2 = false;             // first local steps by the concurrent two-trajectory sweeps
  void* dzs = nullptr;              // [B][Nt+N] per-step overlaps of the sub-interval sweeps (R2)
  void* dckpt = nullptr;            // literal sub-problem: checkpoints, allocated when first needed
  void* dsegb = nullptr;            // literal sub-problem: H1 psi of one segment per (problem, n)
  int cks = 1, nck = 1;             // checkpoint stride and checkpoints per sub-interval
  // dense d = 128, 256 on the tensor cores (ism_tc.cu)
  bool tc = false;
  ism::TcMaps tcmaps{};
  float* dHhi = nullptr;            // TF32 hi / lo parts of [H0; H1], [2d][d]
  float* dHlo = nullptr;
  ism::TcItem* dtc_items = nullptr; // global sweeps: [psi items | chi items], then the sub-interval items
  int tc_npsi = 0, tc_nchi = 0, tc_nsub = 0;   // padded item counts of the three groups
  float* dvstate = nullptr;         // FP32 states of every CTA of the largest launch
  // heterogeneous batch (continuous batching): every row its own problem (ism::RowTab)
  bool het = false;
  int cap = 0;                      // rows allocated; P->B is the number of active rows
  ism::RowTab rt{};
  int hstride = 0;
  void* dzp = nullptr;              // large d: per-step, per-warp overlap partials
  double* du = nullptr;
  float* duf = nullptr;             // FP32 copy of the controls (FP32 propagation)
  double* dgrad = nullptr;
  double* dJn = nullptr;
  double* derr = nullptr;
  double* dJ = nullptr;
  double* dF = nullptr;
  double* dJhist = nullptr;
  double* derrhist = nullptr;
  long hist_cap = 0;
  int* dstatus = nullptr;
  unsigned long long* dcount = nullptr;   // [7]: assembly (3), sub-interval (3), norm drift (double bits)
  bool profiling = false;
  struct Ev { int phase; cudaEvent_t a, b; };
  std::vector<Ev> pending;                // events recorded in the current call
  std::vector<cudaEvent_t> pool;
  double ms[3] = {0, 0, 0};
  long long launches[3] = {0, 0, 0};
  long long kernels = 0;   // every kernel launched, helpers included
  size_t chain_smem = 0;
  int chain_stages = 2;
  size_t bytes = 0;
  std::vector<void*> allocs;
  bool dry = false;   // plan_build for the footprint only: nothing is allocated or uploaded
  bool direct = false;   // d <= 64: global trajectories by direct sweeps instead of assembly + chain
  int sblk = 1, Nc = 0;  // blocked chain: products of sblk consecutive tiles, Nc of them (0: plain)
  void* dMc = nullptr;
};

namespace {

int tc_global(ism_plan_s* P);
int tc_sub(ism_plan_s* P, const ism::KParams& k);

template <class T>
int dalloc(ism_plan_s* P, T** out, size_t count) {
  void* p = nullptr;
  size_t bytes = count * sizeof(T);
  if (bytes == 0) bytes = 16;
  if (P->dry) {   // footprint only: count what would be allocated (cudaMalloc granularity)
    P->bytes += (bytes + 511) / 512 * 512;
    *out = nullptr;
    return ISM_OK;
  }
  // stream-ordered: allocation and release do not synchronise the device, so plans created and
  // destroyed while other plans' kernels run (a serving loop) do not stall them
  cudaError_t e = cudaMallocAsync(&p, bytes, P->st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(e == cudaErrorMemoryAllocation ? ISM_ENOMEM : ISM_ECUDA,
                std::string("cudaMalloc of ") + std::to_string(bytes) + " bytes: " + cudaGetErrorString(e));
  }
  P->allocs.push_back(p);
  P->bytes += (bytes + 511) / 512 * 512;   // the same count as the footprint
  *out = reinterpret_cast<T*>(p);
  return ISM_OK;
}

// The trajectories of the concurrent two-trajectory sweeps are stored per step; above this size the
// first local steps run in k_subfwd instead, which stores one overlap per step.
constexpr size_t kSweeps2MaxBytes = size_t(256) << 20;

// Checkpoints and segment buffer of the literal sub-problem (d <= 64): ceil(ns/S) states (hi + lo in
// FP32 propagation) and S vectors H1 psi per (problem, n).
int alloc_literal(ism_plan_s* P) {
  if (P->dckpt) return ISM_OK;
  const size_t GE = (size_t)P->ks.G * P->ks.E, BN = (size_t)P->B * P->N;
  const size_t parts = P->prec == ISM_FP64 ? 1 : 2;
  unsigned char* c = nullptr;
  unsigned char* sb = nullptr;
  int rc = dalloc(P, &c, BN * P->nck * parts * GE * P->r2);
  if (rc != ISM_OK) return rc;
  rc = dalloc(P, &sb, BN * P->cks * GE * P->r2);
  if (rc != ISM_OK) return rc;
  P->dckpt = c;
  P->dsegb = sb;
  return ISM_OK;
}

void free_all(ism_plan_s* P) {
  for (void* p : P->allocs) cudaFreeAsync(p, P->st);
  P->allocs.clear();
  for (auto& e : P->pending) { cudaEventDestroy(e.a); cudaEventDestroy(e.b); }
  P->pending.clear();
  for (auto e : P->pool) cudaEventDestroy(e);
  P->pool.clear();
}

cudaEvent_t take_event(ism_plan_s* P) {
  if (!P->pool.empty()) { cudaEvent_t e = P->pool.back(); P->pool.pop_back(); return e; }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Launch one phase kernel, bracketed by events when profiling is on.
template <class F>
cudaError_t timed(ism_plan_s* P, int phase, int nkernels, F&& launch) {
  P->launches[phase] += 1;
  P->kernels += nkernels;
  if (!P->profiling) return launch();
  ism_plan_s::Ev ev{phase, take_event(P), take_event(P)};
  cudaEventRecord(ev.a, P->st);
  cudaError_t e = launch();
  cudaEventRecord(ev.b, P->st);
  P->pending.push_back(ev);
  return e;
}

void collect_events(ism_plan_s* P) {
  for (auto& ev : P->pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ev.a, ev.b) == cudaSuccess) P->ms[ev.phase] += ms;
    P->pool.push_back(ev.a);
    P->pool.push_back(ev.b);
  }
  P->pending.clear();
}

}  // namespace

namespace ism {

// Gershgorin enclosures: spec(H0) in [lo, hi], spectral radius of H1 <= h1.
Bounds bounds_of(int kind, int d, const double* H0, const double* H1, const double* H0i, const double* H1i) {
  Bounds b{0, 0, 0};
  b.lo = INFINITY;
  b.hi = -INFINITY;
  if (kind == ISM_H_TRIDIAG) {
    for (int e = 0; e < d; ++e) {
      double r0 = (e > 0 ? std::fabs(H0[d + e - 1]) : 0.0) + (e < d - 1 ? std::fabs(H0[d + e]) : 0.0);
      double r1 = std::fabs(H1[e]) + (e > 0 ? std::fabs(H1[d + e - 1]) : 0.0) + (e < d - 1 ? std::fabs(H1[d + e]) : 0.0);
      b.lo = std::fmin(b.lo, H0[e] - r0);
      b.hi = std::fmax(b.hi, H0[e] + r0);
      b.h1 = std::fmax(b.h1, r1);
    }
  } else if (kind == ISM_H_BITFLIP) {
    int q = 0;
    while (q < 30 && (1 << q) < d) ++q;
    for (int e = 0; e < d; ++e) { b.lo = std::fmin(b.lo, H0[e]); b.hi = std::fmax(b.hi, H0[e]); }
    for (int i = 0; i < q; ++i) b.h1 += std::fabs(H1[i]);
  } else if (kind == ISM_H_PAULI) {   // the controls' bound is taken per sub-interval on the device
    for (int e = 0; e < d; ++e) { b.lo = std::fmin(b.lo, H0[e]); b.hi = std::fmax(b.hi, H0[e]); }
    b.h1 = 1.0;
  } else {   // dense: |H_ef| of the complex entries when imaginary parts are given
    auto mag = [d](const double* re, const double* im, int e, int f) {
      return im ? std::hypot(re[e * d + f], im[e * d + f]) : std::fabs(re[e * d + f]);
    };
    for (int e = 0; e < d; ++e) {
      double r0 = 0.0, r1 = 0.0;
      for (int f = 0; f < d; ++f) {
        if (f != e) r0 += mag(H0, H0i, e, f);
        r1 += mag(H1, H1i, e, f);
      }
      b.lo = std::fmin(b.lo, H0[e * d + e] - r0);
      b.hi = std::fmax(b.hi, H0[e * d + e] + r0);
      b.h1 = std::fmax(b.h1, r1);
    }
  }
  return b;
}

// Device layout of the op data in precision R (see ism_device.cuh).
template <typename R>
std::vector<R> pack_op(int kind, int d, const double* H0, const double* H1, int G, int E, const double* H0i,
                       const double* H1i) {
  std::vector<R> out;
  if (kind == ISM_H_TRIDIAG) {
    out.assign(4 * (size_t)d, R(0));
    for (int e = 0; e < d; ++e) {
      out[e] = (R)H0[e];
      out[2 * d + e] = (R)H1[e];
      if (e < d - 1) { out[d + e] = (R)H0[d + e]; out[3 * d + e] = (R)H1[d + e]; }
    }
  } else if (kind == ISM_H_PAULI) {   // the kernels read the FP64 diagonal and the step coefficients
    out.assign((size_t)d, R(0));
    for (int e = 0; e < d; ++e) out[e] = (R)H0[e];
  } else if (kind == ISM_H_BITFLIP) {
    int q = 0;
    while (q < 30 && (1 << q) < d) ++q;
    out.assign((size_t)d + q, R(0));
    for (int e = 0; e < d; ++e) out[e] = (R)H0[e];
    for (int i = 0; i < q; ++i) out[d + i] = (R)H1[i];
  } else if (H0i || H1i) {   // complex Hermitian: {Re H0, Re H1}, {Im H0, Im H1} per entry
    const int DP = G * E;
    out.assign(4 * (size_t)DP * DP, R(0));
    for (int e = 0; e < d; ++e)
      for (int f = 0; f < d; ++f) {
        R* o = &out[4 * ((size_t)e * DP + f)];
        o[0] = (R)H0[e * d + f];
        o[1] = (R)H1[e * d + f];
        o[2] = H0i ? (R)H0i[e * d + f] : R(0);
        o[3] = H1i ? (R)H1i[e * d + f] : R(0);
      }
  } else {
    const int DP = G * E;
    out.assign(2 * (size_t)DP * DP, R(0));
    for (int e = 0; e < d; ++e)
      for (int f = 0; f < d; ++f) {
        out[2 * ((size_t)e * DP + f)] = (R)H0[e * d + f];
        out[2 * ((size_t)e * DP + f) + 1] = (R)H1[e * d + f];
      }
  }
  return out;
}
template std::vector<float> pack_op<float>(int, int, const double*, const double*, int, int, const double*,
                                           const double*);
template std::vector<double> pack_op<double>(int, int, const double*, const double*, int, int, const double*,
                                             const double*);

// Shape and value checks shared by every entry point that takes an ism_problem.
int validate_problem(const ism_problem& p, int precision) {
  const int d = p.d;
  if (d < 1) return fail(ISM_EINVAL, "d must be >= 1");
  if (p.Nt < 1) return fail(ISM_EINVAL, "Nt must be >= 1");
  if (p.N < 1 || p.N > p.Nt) return fail(ISM_EINVAL, "need 1 <= N <= Nt");
  if (!(p.T > 0.0) || !std::isfinite(p.T)) return fail(ISM_EINVAL, "T must be finite and > 0");
  if (p.batch < 0) return fail(ISM_EINVAL, "batch must be >= 0");
  if (p.kind < ISM_H_DENSE || p.kind > ISM_H_PAULI) return fail(ISM_EINVAL, "unknown Hamiltonian kind");
  if (p.controls < 0 || p.controls > 32 || (p.kind != ISM_H_PAULI && p.controls > 1))
    return fail(ISM_EINVAL, "controls must be 1..32, and 1 unless the kind is ISM_H_PAULI");
  const bool cx = p.H0_imag || p.H1_imag;
  if (cx && p.kind != ISM_H_DENSE) return fail(ISM_EINVAL, "H0_imag and H1_imag apply to the dense kind only");
  if (cx && d > 64) return fail(ISM_EUNSUPPORTED, "complex Hermitian H is built for d <= 64");
  if (p.kind == ISM_H_PAULI) {
    const int m = p.controls < 1 ? 1 : p.controls;
    int q = 0;
    while (q < 30 && (1 << q) < d) ++q;
    if ((1 << q) != d) return fail(ISM_EINVAL, "the Pauli kind needs d = 2^q");
    if (d < 128 || d > 1024) return fail(ISM_EUNSUPPORTED, "this build supports the Pauli kind for d = 128 .. 1024");
    if (!p.H0 || !p.H1 || !p.psi_i || !p.psi_f) return fail(ISM_EINVAL, "H0, H1, psi_i and psi_f are required");
    if (p.objective != ISM_OBJ_OVERLAP) return fail(ISM_EINVAL, "the Pauli kind supports the overlap objective only");
    if (p.alpha) return fail(ISM_EINVAL, "the Pauli kind has no control penalty (alpha must be NULL)");
    if (precision != ISM_FP64 && precision != ISM_MIXED) return fail(ISM_EINVAL, "unknown precision");
    if (!all_finite(p.H0, d) || !all_finite(p.H1, 2L * m * q) || !all_finite(p.psi_i, 2L * d) ||
        !all_finite(p.psi_f, 2L * d))
      return fail(ISM_ENONFINITE, "non-finite value in H0, H1, psi_i or psi_f");
    return ISM_OK;
  }
  if (p.kind == ISM_H_GRID_GP || p.kind == ISM_H_GRID_GP_DOUBLE_WELL) {
    const bool dw = p.kind == ISM_H_GRID_GP_DOUBLE_WELL;
    if (!p.H0 || !p.psi_i || !p.psi_f)
      return fail(ISM_EINVAL, "the grid kinds need H0 = {L, x_min, g} (+ D for the double well), psi_i and psi_f");
    if (p.objective != ISM_OBJ_OVERLAP) return fail(ISM_EINVAL, "the grid kind supports the overlap objective only");
    if (p.alpha) return fail(ISM_EINVAL, "the grid kind has no control penalty (alpha must be NULL)");
    if (precision != ISM_FP64 && precision != ISM_MIXED) return fail(ISM_EINVAL, "unknown precision");
    if (!gp_supported(d)) return fail(ISM_EUNSUPPORTED, "the grid kind supports d = 64 or 512 points");
    if (!all_finite(p.H0, dw ? 4 : 3) || !(p.H0[0] > 0.0) || (dw && !(p.H0[3] > 0.0)))
      return fail(ISM_EINVAL, "grid parameters must be finite with L > 0 (and D > 0)");
    if (!all_finite(p.psi_i, 2L * d) || !all_finite(p.psi_f, 2L * d)) return fail(ISM_ENONFINITE, "non-finite psi_i or psi_f");
    return ISM_OK;
  }
  if (p.objective != ISM_OBJ_OVERLAP && p.objective != ISM_OBJ_OBSERVABLE) return fail(ISM_EINVAL, "unknown objective");
  if (!p.H0 || !p.H1 || !p.psi_i) return fail(ISM_EINVAL, "H0, H1 and psi_i are required");
  if (p.objective == ISM_OBJ_OVERLAP && !p.psi_f) return fail(ISM_EINVAL, "psi_f is required for the overlap objective");
  if (p.objective == ISM_OBJ_OBSERVABLE && !p.O) return fail(ISM_EINVAL, "O is required for the observable objective");
  if (precision != ISM_FP64 && precision != ISM_MIXED) return fail(ISM_EINVAL, "unknown precision");
  int q = 0;
  if (p.kind == ISM_H_BITFLIP) {
    while (q < 30 && (1 << q) < d) ++q;
    if ((1 << q) != d || d < 2) return fail(ISM_EINVAL, "bit-flip kind needs d = 2^q >= 2");
    if (d > 1024) return fail(ISM_EUNSUPPORTED, "this build supports bit-flip d <= 1024");
  } else if (d > 64 && !(p.kind == ISM_H_DENSE && ism::tc_supported(d))) {
    return fail(ISM_EUNSUPPORTED, "this build supports tridiagonal d <= 64 and dense d <= 64, 128 or 256");
  }
  const long nH = p.kind == ISM_H_DENSE ? (long)d * d : p.kind == ISM_H_TRIDIAG ? 2L * d - 1 : d;
  const long nH1 = p.kind == ISM_H_DENSE ? (long)d * d : p.kind == ISM_H_TRIDIAG ? 2L * d - 1 : q;
  if (!all_finite(p.H0, nH) || !all_finite(p.H1, nH1) || !all_finite(p.psi_i, 2L * d))
    return fail(ISM_ENONFINITE, "non-finite value in H0, H1 or psi_i");
  if ((p.H0_imag && !all_finite(p.H0_imag, nH)) || (p.H1_imag && !all_finite(p.H1_imag, nH1)))
    return fail(ISM_ENONFINITE, "non-finite value in H0_imag or H1_imag");
  if (p.objective == ISM_OBJ_OVERLAP && !all_finite(p.psi_f, 2L * d)) return fail(ISM_ENONFINITE, "non-finite psi_f");
  if (p.objective == ISM_OBJ_OBSERVABLE && !all_finite(p.O, (long)d * d)) return fail(ISM_ENONFINITE, "non-finite O");
  if (p.alpha && !all_finite(p.alpha, p.Nt)) return fail(ISM_ENONFINITE, "non-finite alpha");
  // sgn = 1: A = A^T; sgn = -1: A = -A^T (zero diagonal), both to 1e-12 of the largest entry
  auto symmetric = [d](const double* A, double sgn = 1.0) {
    double s = 0.0;
    for (long i = 0; i < (long)d * d; ++i) s = std::fmax(s, std::fabs(A[i]));
    for (int i = 0; i < d; ++i)
      for (int j = 0; j <= i; ++j)
        if (std::fabs(A[i * d + j] - sgn * A[j * d + i]) > 1e-12 * (s + 1e-300)) return false;
    return true;
  };
  if (p.kind == ISM_H_DENSE && (!symmetric(p.H0) || !symmetric(p.H1)))
    return fail(ISM_EINVAL, cx ? "the real parts of dense H0 and H1 must be symmetric" : "dense H0 and H1 must be real symmetric");
  if ((p.H0_imag && !symmetric(p.H0_imag, -1.0)) || (p.H1_imag && !symmetric(p.H1_imag, -1.0)))
    return fail(ISM_EINVAL, "H0_imag and H1_imag must be antisymmetric (H Hermitian)");
  if (p.objective == ISM_OBJ_OBSERVABLE && !symmetric(p.O)) return fail(ISM_EINVAL, "O must be real symmetric");
  return ISM_OK;
}

bool select_kernels(int prec, int kind, int d, KernelSet* ks, bool h1diag, bool cx) {
  if (kind == ISM_H_PAULI) return kernels_pauli(prec, d, ks);
  return kind == ISM_H_TRIDIAG   ? kernels_tridiag(prec, d, h1diag, ks)
         : kind == ISM_H_BITFLIP ? (d > 64 ? kernels_large_bitflip(prec, d, ks) : kernels_bitflip(prec, d, ks))
         : cx                    ? kernels_dense_cx(prec, d, ks)
                                 : kernels_dense(prec, d, ks);
}

void bessel_table(double* out) {
  for (int k = 0; k < 32; ++k) {
    double f = 1.0;
    for (int i = 2; i <= k; ++i) f /= (double)i;   // 1/k!
    out[k * 25] = f;
    for (int m = 1; m <= 24; ++m) out[k * 25 + m] = out[k * 25 + m - 1] / ((double)m * (double)(m + k));
  }
}

}  // namespace ism

namespace {

using ism::Bounds;
using ism::bounds_of;
using ism::pack_op;

int finish(ism_plan_s* P) {
  cudaError_t e = cudaStreamSynchronize(P->st);
  if (e != cudaSuccess) return fail(ISM_ECUDA, std::string("stream: ") + cudaGetErrorString(e));
  collect_events(P);
  int st = 0;
  ISM_CUDA_TRY(cudaMemcpyAsync(&st, P->dstatus, sizeof(int), cudaMemcpyDeviceToHost, P->st));
  ISM_CUDA_TRY(cudaStreamSynchronize(P->st));
  if (st & ism::ST_TIMEOUT) return fail(ISM_ETIMEOUT, "a bounded device-side wait gave up");
  const bool cn = P->scheme == ISM_SCHEME_CRANK_NICOLSON;
  if (st & ism::ST_KOVERFLOW) return fail(ISM_EUNSUPPORTED, "Chebyshev series needed more terms than compiled");
  if (st & ism::ST_NONFINITE) return fail(ISM_ENONFINITE, "non-finite value in a control or a result");
  if (st & ism::ST_SPECTRUM)
    return fail(ISM_EUNSUPPORTED, cn ? "controls so large that tau/2 times the off-diagonal row sum of H reaches 1/2 "
                                       "(the Jacobi solve of the Crank-Nicolson step)"
                                     : "controls so large that a time step needs more Chebyshev sub-steps than the limit");
  g_err.clear();
  return ISM_OK;
}

int begin(ism_plan_s* P) {
  ISM_CUDA_TRY(cudaSetDevice(P->dev));
  ISM_CUDA_TRY(cudaMemsetAsync(P->dstatus, 0, sizeof(int), P->st));
  return ISM_OK;
}

ism::KParams kparams(ism_plan_s* P, double* u) {
  ism::KParams k{};
  k.d = P->d; k.Nt = P->Nt; k.N = P->N; k.B = P->B; k.ldm = P->ldm; k.dpad = P->dpad; k.tile_stride = P->tst;
  k.tau = P->tau; k.T = P->T; k.c0 = P->c0; k.r0 = P->r0; k.h1n = P->h1n; k.tol = P->tol;
  k.rho = P->rho; k.w = P->w;
  k.jn = P->djn; k.beta = P->dbeta; k.alpha = P->dalpha; k.H = P->dH; k.H0d = P->dH0d;
  k.cheb = P->dcheb; k.ctab = P->dctab; k.pen = P->dpen; k.phase = P->dphase;
  k.u = u; k.phi = P->dphi; k.M = P->dM; k.traj = P->dtraj; k.traj2 = P->dtraj2;
  k.zs = P->dzs; k.ckpt = P->dckpt; k.segb = P->dsegb; k.cks = P->cks; k.nck = P->nck;
  k.grad = P->dgrad; k.Jn = P->dJn; k.err = P->derr; k.status = P->dstatus;
  k.count = P->dcount;
  k.psin = P->dpsin; k.chin = P->dchin; k.form = 0;
  k.update = 0; k.max_spin = P->max_spin;
  k.psi_i = P->dpsi_i; k.psi_f = P->dpsi_f; k.O = P->dO; k.obj = P->obj; k.uf = P->duf;
  k.psin_w = P->dpsin; k.chin_w = P->dchin; k.zp = P->dzp;
  k.scheme = P->scheme == ISM_SCHEME_CRANK_NICOLSON ? 1 : 0;
  k.m = P->m; k.q = P->q; k.wts = P->dwts; k.cxy = P->dcxy; k.zq = P->dzp;
  k.nrm_w = P->dnrm;
  k.het = P->het ? 1 : 0;
  k.rt = P->rt;
  return k;
}

// The per-sub-interval parameters of the plan's kernels at the controls of k.
cudaError_t prep_params(ism_plan_s* P, const ism::KParams& k) {
  return P->ks.prep ? P->ks.prep(k, P->st) : ism::launch_cheb_prep(P->prec, k, P->st);
}

ism::GPParams gparams(ism_plan_s* P, double* u) {
  ism::GPParams g{};
  g.n = P->d; g.Nt = P->Nt; g.N = P->N; g.B = P->B;
  g.tau = P->tau; g.T = P->T; g.L = P->gpL; g.xmin = P->gpxmin; g.dx = P->gpL / P->d; g.g = P->gpg; g.rho = P->rho;
  g.pot = P->gppot; g.dw = P->gpdw;
  g.jn = P->djn; g.u = u; g.psi_i = P->dpsi_i; g.psi_f = P->dpsi_f; g.traj = P->dtraj;
  g.cks = P->cks; g.nck = P->nck; g.gck = P->dckpt; g.segb = P->dsegb; g.tab = P->dgptab;
  g.psin = P->dpsin; g.chin = P->dchin; g.grad = P->dgrad; g.Jn = P->dJn; g.err = P->derr;
  g.J = P->dJ; g.F = P->dF; g.Jhist = nullptr; g.hist_stride = 0; g.hist_k = 0;
  g.status = P->dstatus; g.count = P->dcount; g.update = 0; g.reuse = 0;
  return g;
}

// a-b of Algorithm 1: assemble M_n, chain, phi, J/F (optionally into Jhist[.][hist_k]).
int run_states(ism_plan_s* P, const double* u, double* Jhist, int hist_stride, int hist_k) {
  if (P->gp) {   // nonlinear: sequential forward sweep (psi(t_n), J) then adjoint sweep (chi(t_n))
    ism::GPParams g = gparams(P, const_cast<double*>(u));
    g.Jhist = Jhist; g.hist_stride = hist_stride; g.hist_k = hist_k;
    ISM_CUDA_TRY(timed(P, 0, 1, [&] { return ism::launch_gp_forward(P->prec, g, P->st); }));
    g.count = P->dcount + 1;
    ISM_CUDA_TRY(timed(P, 1, 1, [&] { return ism::launch_gp_adjoint(P->prec, g, P->st); }));
    return ISM_OK;
  }
  ism::KParams k = kparams(P, const_cast<double*>(u));
  if (P->tc) {   // dense d = 128, 256: the stacked global sweeps on the tensor cores
    ISM_CUDA_TRY(prep_params(P, k));
    P->kernels += 1;
    int rc = tc_global(P);
    if (rc != ISM_OK) return rc;
  } else if (P->ks.large || P->direct) {   // direct sweeps: psi(t_n), chi(t_n) in FP64
    ism::LaunchFn sweep = P->ks.large ? P->ks.lsweep : P->wide ? P->ks.gsweep_wide : P->ks.gsweep;
    ISM_CUDA_TRY(timed(P, 0, 2, [&] {
      cudaError_t e = prep_params(P, k);
      return e != cudaSuccess ? e : sweep(k, P->st);
    }));
  } else {
    ISM_CUDA_TRY(timed(P, 0, 2, [&] {
      cudaError_t e = prep_params(P, k);
      return e != cudaSuccess ? e : P->ks.assemble(k, P->st);
    }));
  }
  ism::ChainParams c{};
  c.d = P->d; c.Nt = P->Nt; c.N = P->N; c.B = P->B; c.ldm = P->ldm; c.obj = P->obj;
  c.tau = P->tau; c.T = P->T; c.M = P->dM; c.psi_i = P->dpsi_i; c.psi_f = P->dpsi_f; c.O = P->dO;
  c.alpha = P->dalpha; c.u = u; c.jn = P->djn; c.ab = P->dab; c.stage = P->dstage;
  c.pen = P->dalpha ? P->dpen : nullptr; c.psin = P->dpsin; c.chin = P->dchin; c.phi = P->dphi;
  c.J = P->dJ; c.F = P->dF; c.Jhist = Jhist; c.hist_stride = hist_stride; c.hist_k = hist_k;
  c.status = P->dstatus; c.max_spin = P->max_spin; c.stages = P->chain_stages; c.tile_stride = P->tst;
  c.Mc = P->dMc; c.Nc = P->Nc; c.sblk = P->sblk;
  c.drift = P->dcount + 6;
  c.nrm_psi_i = P->nrm_psi_i;
  c.inv_nrm_psi_i = P->nrm_psi_i > 0.0 ? 1.0 / P->nrm_psi_i : 0.0;
  c.nrm_chi_T = P->obj == ISM_OBJ_OVERLAP ? P->nrm_psi_f : -1.0;
  c.nrm = (P->direct && !P->ks.large) ? P->dnrm : nullptr;   // k_gsweep leaves the squared norms
  c.het = P->het ? 1 : 0;
  c.rt = P->rt;
  if (P->ks.large || P->direct || P->tc) {
    c.src64 = 1;
    ISM_CUDA_TRY(timed(P, 1, 1, [&] { return ism::launch_phi(P->prec, c, P->st); }));
  } else {
    ISM_CUDA_TRY(timed(P, 1, P->Nc ? 4 : 2, [&] { return ism::launch_chain(P->prec, c, P->chain_smem, P->st); }));
  }
  return ISM_OK;
}

// Bring a caller array of n doubles to the device: device pointers are used in place, host data is
// copied into `staging` after a finiteness check.
int stage_in(ism_plan_s* P, const double* src, long n, double* staging, const double** out, bool check) {
  if (is_device_ptr(src)) {
    if (check) {
      int blocks = (int)std::min<long>(1024, (n + 255) / 256);
      if (blocks < 1) blocks = 1;
      ism::k_check_finite<<<blocks, 256, 0, P->st>>>(src, n, P->dstatus);
      P->kernels += 1;
      ISM_CUDA_TRY(cudaGetLastError());
    }
    *out = src;
    return ISM_OK;
  }
  // host data: copy, then check on the device (a host pass over a large batch of controls would
  // cost more than the copy); a non-finite value surfaces as ISM_ENONFINITE when the call finishes
  ISM_CUDA_TRY(cudaMemcpyAsync(staging, src, n * sizeof(double), cudaMemcpyHostToDevice, P->st));
  if (check) {
    int blocks = (int)std::min<long>(1024, (n + 255) / 256);
    if (blocks < 1) blocks = 1;
    ism::k_check_finite<<<blocks, 256, 0, P->st>>>(staging, n, P->dstatus);
    P->kernels += 1;
    ISM_CUDA_TRY(cudaGetLastError());
  }
  *out = staging;
  return ISM_OK;
}

int copy_out(ism_plan_s* P, double* dst, const void* src, long n) {
  if (!dst) return ISM_OK;
  ISM_CUDA_TRY(cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDefault, P->st));
  return ISM_OK;
}

int ensure_hist(ism_plan_s* P, long cap) {
  if (cap <= P->hist_cap) return ISM_OK;
  // old buffers stay in the plan's list and are freed at destroy
  int rc = dalloc(P, &P->dJhist, (size_t)P->B * cap);
  if (rc) return rc;
  rc = dalloc(P, &P->derrhist, (size_t)P->B * cap);
  if (rc) return rc;
  P->hist_cap = cap;
  return ISM_OK;
}

}  // namespace

extern "C" {

const char* ism_last_error(void) { return g_err.c_str(); }

const char* ism_version(void) { return "ism-gb300 0.1 (sm_103a)"; }

}  // extern "C"

namespace {

// TF32 rounding of an FP32 value (round half away from zero on the 13 dropped mantissa bits).
float tf32_round(float x) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  u = (u + 0x1000u) & 0xFFFFE000u;
  float r;
  std::memcpy(&r, &u, 4);
  return r;
}

// Dense d = 128, 256: [H0; H1] as TF32 hi + lo parts, the stacked states of the global and the
// sub-interval sweeps, and the plan's FP64 arrays.  Mixed precision and one local step only.
int plan_build_tc(ism_plan_s* P, const ism_problem& p, bool dry, size_t* bytes_out) {
  const int d = p.d;
  if (P->prec != ISM_MIXED)
    return fail(ISM_EUNSUPPORTED, "dense d = 128 and 256 run on the tensor cores in mixed precision only");
  if (P->L != 1) return fail(ISM_EUNSUPPORTED, "dense d = 128 and 256 support one local step per iteration");
  P->tc = true;
  P->form = 2;
  P->cks = P->nck = 0;   // no literal sub-problems: nothing is checkpointed
  P->r2 = sizeof(float2);
  {
    Bounds bd = bounds_of(ISM_H_DENSE, d, p.H0, p.H1);
    P->c0 = 0.5 * (bd.lo + bd.hi);
    P->r0 = 0.5 * (bd.hi - bd.lo);
    P->h1n = bd.h1;
  }
  std::vector<int> jn;
  std::vector<double> beta;
  std::vector<double2> phase;
  ism::partition(P->T, P->Nt, P->N, P->c0, &jn, &beta, &phase);
  const int NI = ism::tc_items_per_cta(d);
  const size_t B = P->B;
  auto pad = [NI](int n) { return (n + NI - 1) / NI * NI; };
  P->tc_npsi = pad(P->B);
  P->tc_nchi = pad(P->B);
  P->tc_nsub = pad(2 * P->B * P->N);
  const int ctas = std::max((P->obj == ISM_OBJ_OVERLAP ? P->tc_npsi + P->tc_nchi : P->tc_npsi), P->tc_nsub) / NI;
  int rc = ISM_OK;
#define TRY_TC(ptr, n) if ((rc = dalloc(P, &(ptr), (n))) != ISM_OK) return rc;
  TRY_TC(P->dHhi, 2 * (size_t)d * d);
  TRY_TC(P->dHlo, 2 * (size_t)d * d);
  TRY_TC(P->djn, (size_t)P->N + 1);
  TRY_TC(P->dbeta, (size_t)P->N);
  TRY_TC(P->dab, (size_t)P->N + 1);
  TRY_TC(P->dphase, (size_t)P->N);
  TRY_TC(P->dcheb, B * P->N * ism::cheb_bytes(ISM_MIXED));
  TRY_TC(P->dpen, B * P->N);
  TRY_TC(P->dctab, (size_t)ism::BESSEL_TABLE);
  if (p.alpha) TRY_TC(P->dalpha, (size_t)P->Nt);
  TRY_TC(P->dpsi_i, (size_t)d);
  TRY_TC(P->dpsi_f, (size_t)d);
  if (p.objective == ISM_OBJ_OBSERVABLE) TRY_TC(P->dO, (size_t)d * d);
  TRY_TC(P->dpsin, B * (P->N + 1) * (size_t)d);
  TRY_TC(P->dchin, B * (P->N + 1) * (size_t)d);
  TRY_TC(P->dphi, B * (P->N + 1) * (size_t)d);
  {
    unsigned char* dZ = nullptr;
    TRY_TC(dZ, B * ((size_t)P->Nt + P->N) * sizeof(float2));
    P->dzs = dZ;
  }
  TRY_TC(P->du, B * P->Nt);
  TRY_TC(P->duf, B * P->Nt);
  TRY_TC(P->dgrad, B * P->Nt);
  TRY_TC(P->dJn, B * P->N);
  TRY_TC(P->derr, B * P->N);
  TRY_TC(P->dJ, B);
  TRY_TC(P->dF, B);
  TRY_TC(P->dstatus, 1);
  TRY_TC(P->dcount, 7);
  TRY_TC(P->dtc_items, (size_t)P->tc_npsi + P->tc_nchi + P->tc_nsub);
  TRY_TC(P->dvstate, (size_t)ctas * 2 * (2 * NI) * d);
#undef TRY_TC
  if (dry) {
    *bytes_out = P->bytes;
    return ISM_OK;
  }
  // [H0; H1] rows as TF32 hi + lo (the tensor cores read the top 19 bits of each word)
  std::vector<float> hi(2 * (size_t)d * d), lo(2 * (size_t)d * d);
  for (int m = 0; m < 2 * d; ++m)
    for (int e = 0; e < d; ++e) {
      const double x = m < d ? p.H0[(size_t)m * d + e] : p.H1[(size_t)(m - d) * d + e];
      const float h = tf32_round((float)x);
      hi[(size_t)m * d + e] = h;
      lo[(size_t)m * d + e] = tf32_round((float)(x - (double)h));
    }
  std::vector<ism::TcItem> items((size_t)P->tc_npsi + P->tc_nchi + P->tc_nsub, ism::TcItem{-1, 0, 0, 0});
  for (int b = 0; b < P->B; ++b) {
    items[b] = ism::TcItem{b, 0, 0, 0};
    items[P->tc_npsi + b] = ism::TcItem{b, 0, 0, 1};
  }
  for (int b = 0; b < P->B; ++b)
    for (int n = 0; n < P->N; ++n)
      for (int r = 0; r < 2; ++r)
        items[(size_t)P->tc_npsi + P->tc_nchi + 2 * ((size_t)b * P->N + n) + r] = ism::TcItem{b, n, r, 0};
  cudaError_t e = cudaSuccess;
  auto h2d = [&](void* dst, const void* src, size_t n) {
    if (e == cudaSuccess) e = cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, P->st);
  };
  h2d(P->dHhi, hi.data(), hi.size() * sizeof(float));
  h2d(P->dHlo, lo.data(), lo.size() * sizeof(float));
  h2d(P->djn, jn.data(), jn.size() * sizeof(int));
  h2d(P->dbeta, beta.data(), beta.size() * sizeof(double));
  h2d(P->dphase, phase.data(), phase.size() * sizeof(double2));
  std::vector<double2> ab(P->N + 1);
  for (int n = 0; n <= P->N; ++n) {
    const double tn = jn[n] * P->tau;
    ab[n] = make_double2((P->T - tn) / P->T, tn / P->T);
  }
  h2d(P->dab, ab.data(), ab.size() * sizeof(double2));
  std::vector<double> tab(ism::BESSEL_TABLE);
  ism::bessel_table(tab.data());
  h2d(P->dctab, tab.data(), tab.size() * sizeof(double));
  if (p.alpha) h2d(P->dalpha, p.alpha, P->Nt * sizeof(double));
  h2d(P->dpsi_i, p.psi_i, 2 * sizeof(double) * d);
  if (p.objective == ISM_OBJ_OVERLAP) h2d(P->dpsi_f, p.psi_f, 2 * sizeof(double) * d);
  else if (e == cudaSuccess) e = cudaMemsetAsync(P->dpsi_f, 0, 2 * sizeof(double) * d, P->st);
  if (p.objective == ISM_OBJ_OBSERVABLE) h2d(P->dO, p.O, sizeof(double) * d * d);
  h2d(P->dtc_items, items.data(), items.size() * sizeof(ism::TcItem));
  if (e == cudaSuccess) e = cudaMemsetAsync(P->dstatus, 0, sizeof(int), P->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(P->dcount, 0, 7 * sizeof(unsigned long long), P->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(P->st);   // the host arrays above are local
  if (e == cudaSuccess) e = ism::tc_encode_maps(&P->tcmaps, P->dHhi, P->dHlo, d);
  if (e != cudaSuccess) return fail(ISM_ECUDA, std::string("plan upload: ") + cudaGetErrorString(e));
  for (int e0 = 0; e0 < d; ++e0) {
    P->nrm_psi_i += p.psi_i[2 * e0] * p.psi_i[2 * e0] + p.psi_i[2 * e0 + 1] * p.psi_i[2 * e0 + 1];
    if (p.objective == ISM_OBJ_OVERLAP)
      P->nrm_psi_f += p.psi_f[2 * e0] * p.psi_f[2 * e0] + p.psi_f[2 * e0 + 1] * p.psi_f[2 * e0 + 1];
  }
  return ISM_OK;
}

// The stacked tensor-core sweeps of a dense d = 128, 256 plan.  mode 0: psi forward and chi backward
// (Algorithm 1 (a)-(b)); mode 1: the sub-problems of every (problem, n) in the two-trajectory form.
ism::TcParams tc_params(ism_plan_s* P, int mode) {
  ism::TcParams t{};
  t.d = P->d; t.Nt = P->Nt; t.N = P->N; t.B = P->B; t.obj = P->obj; t.mode = mode;
  t.nsteps = mode == 0 ? P->Nt : (P->Nt + P->N - 1) / P->N;
  t.jn = P->djn; t.uf = P->duf; t.cheb = P->dcheb;
  t.psi_i = P->dpsi_i; t.psi_f = P->dpsi_f; t.psin = P->dpsin; t.chin = P->dchin;
  t.zs = reinterpret_cast<float2*>(P->dzs);
  t.vstate = P->dvstate;
  t.status = P->dstatus;
  t.max_spin = P->max_spin;
  t.count = P->dcount + (mode == 0 ? 0 : 3);
  return t;
}

int tc_global(ism_plan_s* P) {
  ism::TcParams t = tc_params(P, 0);
  if (P->obj == ISM_OBJ_OVERLAP) {   // psi forward and chi backward together
    t.items = P->dtc_items;
    t.nitems = P->tc_npsi + P->tc_nchi;
    ISM_CUDA_TRY(timed(P, 0, 1, [&] { return ism::launch_tc_sweep(P->tcmaps, t, P->st); }));
    return ISM_OK;
  }
  t.items = P->dtc_items;            // observable: psi, then chi(T) = O psi(T), then chi
  t.nitems = P->tc_npsi;
  ISM_CUDA_TRY(timed(P, 0, 1, [&] { return ism::launch_tc_sweep(P->tcmaps, t, P->st); }));
  ISM_CUDA_TRY(ism::launch_tc_chiT(P->dO, P->dpsin, P->dchin, P->d, P->N, P->B, P->st));
  P->kernels += 1;
  t.items = P->dtc_items + P->tc_npsi;
  t.nitems = P->tc_nchi;
  ISM_CUDA_TRY(timed(P, 0, 1, [&] { return ism::launch_tc_sweep(P->tcmaps, t, P->st); }));
  return ISM_OK;
}

// step (c) of a dense d = 128, 256 plan: the stacked sub-interval sweep, then the FP64 gradient pass
int tc_sub(ism_plan_s* P, const ism::KParams& k) {
  ism::TcParams t = tc_params(P, 1);
  t.items = P->dtc_items + P->tc_npsi + P->tc_nchi;
  t.nitems = P->tc_nsub;
  ISM_CUDA_TRY(timed(P, 2, 2, [&] {
    cudaError_t e = ism::launch_tc_sweep(P->tcmaps, t, P->st);
    return e != cudaSuccess ? e : ism::launch_tc_zgrad(k, P->st);
  }));
  return ISM_OK;
}

// Validate, size and (unless dry) allocate and upload a plan.  dry: only *bytes is produced.
int plan_build(const ism_problem* prob, const ism_options* opt, void* cuda_stream, ism_plan_t* out, bool dry,
               size_t* bytes_out) {
  if (!prob || !opt || (!out && !dry)) return fail(ISM_EINVAL, "null problem, options or output handle");
  const ism_problem& p = *prob;
  const int d = p.d;
  {
    int rc0 = ism::validate_problem(p, opt->precision);
    if (rc0 != ISM_OK) return rc0;
  }
  if (opt->local_iters < 0) return fail(ISM_EINVAL, "local_iters must be >= 1");
  if (!(opt->rho >= 0.0) || !std::isfinite(opt->rho)) return fail(ISM_EINVAL, "rho must be finite and >= 0");
  if (opt->cheb_tol < 0.0) return fail(ISM_EINVAL, "cheb_tol must be >= 0");
  if (opt->subproblem_form < 0 || opt->subproblem_form > 2) return fail(ISM_EINVAL, "subproblem_form must be 0, 1 or 2");
  if (opt->step1 < 0 || opt->step1 > 2) return fail(ISM_EINVAL, "step1 must be 0, 1 or 2");
  if (opt->ckpt_stride < 0) return fail(ISM_EINVAL, "ckpt_stride must be >= 0");
  if (opt->scheme != ISM_SCHEME_CHEBYSHEV && opt->scheme != ISM_SCHEME_CRANK_NICOLSON)
    return fail(ISM_EINVAL, "scheme must be ISM_SCHEME_CHEBYSHEV or ISM_SCHEME_CRANK_NICOLSON");
  if (opt->scheme == ISM_SCHEME_CRANK_NICOLSON &&
      (p.kind == ISM_H_GRID_GP || p.kind == ISM_H_GRID_GP_DOUBLE_WELL || p.kind == ISM_H_PAULI || p.d > 64))
    return fail(ISM_EUNSUPPORTED, "the Crank-Nicolson scheme is built for the tridiagonal, dense and bit-flip kinds "
                                  "with d <= 64");
  if (opt->scheme == ISM_SCHEME_CRANK_NICOLSON && (p.H0_imag || p.H1_imag))
    return fail(ISM_EUNSUPPORTED, "the Crank-Nicolson scheme is built for real symmetric H");

  ism_plan_s* P = new (std::nothrow) ism_plan_s();
  if (!P) return fail(ISM_ENOMEM, "host allocation");
  P->dry = dry;
  P->d = d; P->kind = p.kind; P->obj = p.objective; P->Nt = p.Nt; P->N = p.N; P->B = p.batch < 1 ? 1 : p.batch;
  P->prec = opt->precision; P->L = opt->local_iters < 1 ? 1 : opt->local_iters;
  P->T = p.T; P->tau = p.T / p.Nt; P->rho = opt->rho;
  P->tol = opt->cheb_tol > 0 ? opt->cheb_tol : (P->prec == ISM_FP64 ? 1e-17 : 1e-10);
  P->w = p.objective == ISM_OBJ_OVERLAP ? 1.0 : 2.0;
  P->max_spin = opt->max_spin_iters > 0 ? opt->max_spin_iters : (1 << 22);
  P->form = opt->subproblem_form != 0 ? opt->subproblem_form : 2;
  P->scheme = opt->scheme;
  P->st = reinterpret_cast<cudaStream_t>(cuda_stream);
  cudaGetDevice(&P->dev);

  if (p.kind == ISM_H_DENSE && ism::tc_supported(d)) {   // dense d = 128, 256: the tensor-core path
    int rc0 = plan_build_tc(P, p, dry, bytes_out);
    if (rc0 != ISM_OK || dry) { if (!dry || rc0 != ISM_OK) { free_all(P); } delete P; return rc0; }
    *out = P;
    g_err.clear();
    return ISM_OK;
  }
  if (p.kind == ISM_H_GRID_GP || p.kind == ISM_H_GRID_GP_DOUBLE_WELL) {
    P->gp = true;
    P->gpL = p.H0[0];
    P->gpxmin = p.H0[1];
    P->gpg = p.H0[2];
    P->gppot = p.kind == ISM_H_GRID_GP_DOUBLE_WELL ? 1 : 0;
    P->gpdw = P->gppot ? p.H0[3] : 0.0;
    P->r2 = P->prec == ISM_FP64 ? sizeof(double2) : sizeof(float2);
    std::vector<int> jn;
    ism::partition(P->T, P->Nt, P->N, 0.0, &jn, nullptr, nullptr);
    int rc = ISM_OK;
    const size_t B = P->B;
#define TRY_GP(ptr, n) if ((rc = dalloc(P, &(ptr), (n))) != ISM_OK) { free_all(P); delete P; return rc; }
    // the forward states the adjoint sweeps read: the whole trajectory, or (ckpt_stride S > 0) the
    // states every S steps of each sub-interval plus one S-step segment per (problem, sub-interval)
    if (opt->ckpt_stride > 0) {
      const int nsmax = (P->Nt + P->N - 1) / P->N;
      P->cks = opt->ckpt_stride > nsmax ? nsmax : opt->ckpt_stride;
      P->nck = (nsmax + P->cks - 1) / P->cks;
      unsigned char* dC = nullptr;
      TRY_GP(dC, B * P->N * (size_t)P->nck * d * P->r2);
      P->dckpt = dC;
      unsigned char* dS = nullptr;
      TRY_GP(dS, B * P->N * (size_t)P->cks * d * P->r2);
      P->dsegb = dS;
    } else {
      P->cks = P->nck = 0;
      unsigned char* dTb = nullptr;
      TRY_GP(dTb, B * ((size_t)P->Nt + 1) * d * P->r2);
      P->dtraj = dTb;
    }
    TRY_GP(P->djn, (size_t)P->N + 1);
    TRY_GP(P->dpsi_i, (size_t)d);
    TRY_GP(P->dpsi_f, (size_t)d);
    TRY_GP(P->dpsin, B * (P->N + 1) * (size_t)d);
    TRY_GP(P->dchin, B * (P->N + 1) * (size_t)d);
    TRY_GP(P->du, B * P->Nt);
    TRY_GP(P->dgrad, B * P->Nt);
    TRY_GP(P->dJn, B * P->N);
    TRY_GP(P->derr, B * P->N);
    TRY_GP(P->dJ, B);
    TRY_GP(P->dF, B);
    TRY_GP(P->dstatus, 1);
    TRY_GP(P->dcount, 7);
    {
      unsigned char* dT = nullptr;
      TRY_GP(dT, ism::gp_table_bytes(P->prec == ISM_FP64 ? 0 : 1, d));
      P->dgptab = dT;
    }
#undef TRY_GP
    if (dry) {
      *bytes_out = P->bytes;
      delete P;
      return ISM_OK;
    }
    cudaError_t e = cudaMemcpyAsync(P->djn, jn.data(), jn.size() * sizeof(int), cudaMemcpyHostToDevice, P->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(P->dpsi_i, p.psi_i, 2 * sizeof(double) * d, cudaMemcpyHostToDevice, P->st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(P->dpsi_f, p.psi_f, 2 * sizeof(double) * d, cudaMemcpyHostToDevice, P->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(P->dstatus, 0, sizeof(int), P->st);
    if (e == cudaSuccess) e = cudaMemsetAsync(P->dcount, 0, 7 * sizeof(unsigned long long), P->st);
    if (e == cudaSuccess) {   // the plan's tables (n, L, tau, x_min are fixed for its life)
      ism::GPParams g = gparams(P, P->du);
      e = ism::launch_gp_tables(P->prec == ISM_FP64 ? 0 : 1, g, P->st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(P->st);   // the host arrays above are local
    if (e != cudaSuccess) {
      free_all(P);
      delete P;
      return fail(ISM_ECUDA, std::string("plan upload: ") + cudaGetErrorString(e));
    }
    *out = P;
    g_err.clear();
    return ISM_OK;
  }

  for (int e = 0; e < d; ++e) {
    P->nrm_psi_i += p.psi_i[2 * e] * p.psi_i[2 * e] + p.psi_i[2 * e + 1] * p.psi_i[2 * e + 1];
    if (p.objective == ISM_OBJ_OVERLAP && p.psi_f)
      P->nrm_psi_f += p.psi_f[2 * e] * p.psi_f[2 * e] + p.psi_f[2 * e + 1] * p.psi_f[2 * e + 1];
  }
  if (p.kind == ISM_H_PAULI) {
    P->pauli = true;
    P->m = p.controls < 1 ? 1 : p.controls;
    while (P->q < 30 && (1 << P->q) < d) ++P->q;
  }
  bool h1diag = true;
  if (p.kind == ISM_H_TRIDIAG) {
    h1diag = false;
    for (int e = 0; e < d; ++e) h1diag |= p.H1[e] != 0.0;
  }
  bool ok = P->scheme == ISM_SCHEME_CRANK_NICOLSON ? ism::kernels_cn(P->prec, p.kind, d, h1diag, &P->ks)
                                                    : ism::select_kernels(P->prec, p.kind, d, &P->ks, h1diag,
                                                                          p.H0_imag || p.H1_imag);
  if (!ok) { delete P; return fail(ISM_EUNSUPPORTED, "no compiled kernel for this kind and d"); }
  P->direct = !P->ks.large && (opt->step1 == 2 || (opt->step1 == 0 && P->B >= 96));
  if (P->direct && P->ks.gsweep_wide) {
    // the wide layout holds 128 / GW problems per CTA; it pays once every SM gets two of its CTAs
    int nsm = 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, P->dev) != cudaSuccess || nsm < 1) {
      cudaGetLastError();
      nsm = 152;
    }
    P->wide = (long)P->B >= 2L * nsm * (128 / P->ks.GW);
  }
  const int gpw = P->ks.large ? 1 : 32 / P->ks.GA;
  P->dpad = (d + gpw - 1) / gpw * gpw;
  P->ldm = d | 1;                                   // odd column stride
  P->tst = ((long)d * P->ldm + 1) / 2 * 2;          // even tile stride: tiles are multiples of 16 bytes
  P->r2 = P->prec == ISM_FP64 ? sizeof(double2) : sizeof(float2);

  if (P->scheme == ISM_SCHEME_CRANK_NICOLSON) {
    // no centring (c0 = 0: no segment phase); r0, h1n = largest off-diagonal absolute row sums of H0,
    // H1, which bound the contraction of the Jacobi solve
    P->c0 = 0.0;
    P->r0 = P->h1n = 0.0;
    if (p.kind == ISM_H_TRIDIAG) {
      for (int e = 0; e < d; ++e) {
        const double l0 = e > 0 ? std::fabs(p.H0[d + e - 1]) : 0.0, r0 = e < d - 1 ? std::fabs(p.H0[d + e]) : 0.0;
        const double l1 = e > 0 ? std::fabs(p.H1[d + e - 1]) : 0.0, r1 = e < d - 1 ? std::fabs(p.H1[d + e]) : 0.0;
        P->r0 = std::fmax(P->r0, l0 + r0);
        P->h1n = std::fmax(P->h1n, l1 + r1);
      }
    } else if (p.kind == ISM_H_BITFLIP) {   // H0 diagonal; every row of H1 holds |h_i| once per flip
      int q = 0;
      while (q < 30 && (1 << q) < d) ++q;
      for (int i = 0; i < q; ++i) P->h1n += std::fabs(p.H1[i]);
    } else {   // dense
      for (int e = 0; e < d; ++e) {
        double s0 = 0.0, s1 = 0.0;
        for (int f = 0; f < d; ++f)
          if (f != e) { s0 += std::fabs(p.H0[(size_t)e * d + f]); s1 += std::fabs(p.H1[(size_t)e * d + f]); }
        P->r0 = std::fmax(P->r0, s0);
        P->h1n = std::fmax(P->h1n, s1);
      }
    }
  } else {
    Bounds bd = bounds_of(p.kind, d, p.H0, p.H1, p.H0_imag, p.H1_imag);
    P->c0 = 0.5 * (bd.lo + bd.hi);
    P->r0 = 0.5 * (bd.hi - bd.lo);
    P->h1n = bd.h1;
  }

  // partition (Sec. 2): j_n = floor(n Nt / N), t_n = j_n tau, beta_n = T / (t_{n+1} - t_n)
  std::vector<int> jn;
  std::vector<double> beta;
  std::vector<double2> phase;   // the global phase of each segment, once per plan
  ism::partition(P->T, P->Nt, P->N, P->c0, &jn, &beta, &phase);

  int rc = ISM_OK;
  const int GE = P->ks.G * P->ks.E;
  const size_t B = P->B;
#define TRY_ALLOC(ptr, n) if ((rc = dalloc(P, &(ptr), (n))) != ISM_OK) { free_all(P); delete P; return rc; }
  unsigned char* dHb = nullptr;
  size_t hbytes;
  std::vector<double> hd;
  std::vector<float> hf;
  if (P->prec == ISM_FP64) {
    hd = pack_op<double>(p.kind, d, p.H0, p.H1, P->ks.G, P->ks.E, p.H0_imag, p.H1_imag);
    hbytes = hd.size() * sizeof(double);
  } else {
    hf = pack_op<float>(p.kind, d, p.H0, p.H1, P->ks.G, P->ks.E, p.H0_imag, p.H1_imag);
    hbytes = hf.size() * sizeof(float);
  }
  TRY_ALLOC(dHb, hbytes);
  P->dH = dHb;
  TRY_ALLOC(P->dH0d, (size_t)d);
  TRY_ALLOC(P->djn, (size_t)P->N + 1);
  TRY_ALLOC(P->dbeta, (size_t)P->N);
  TRY_ALLOC(P->dab, (size_t)P->N + 1);
  TRY_ALLOC(P->dphase, (size_t)P->N);
  TRY_ALLOC(P->dcheb, B * P->N * ism::cheb_bytes(P->prec));
  if (!P->ks.large && !P->direct) TRY_ALLOC(P->dstage, B * 2 * ((size_t)P->N + 1) * d * P->r2);
  TRY_ALLOC(P->dpen, B * P->N);
  TRY_ALLOC(P->dctab, (size_t)ism::BESSEL_TABLE);
  if (p.alpha) TRY_ALLOC(P->dalpha, (size_t)P->Nt);
  TRY_ALLOC(P->dpsi_i, (size_t)d);
  TRY_ALLOC(P->dpsi_f, (size_t)d);
  if (p.objective == ISM_OBJ_OBSERVABLE) TRY_ALLOC(P->dO, (size_t)d * d);
  if (!P->ks.large && !P->direct) {   // sub-interval propagators M_n (assembly + chain)
    unsigned char* dMb = nullptr;
    TRY_ALLOC(dMb, B * P->N * (size_t)P->tst * P->r2);
    P->dM = dMb;
    // blocked chain from N = 32: blocks of ~sqrt(N) tiles, as many as fit in shared memory
    const size_t tile = (size_t)P->tst * P->r2;
    int sb = (int)std::lround(std::sqrt((double)P->N));
    while (sb > 1 && (sb * tile > 200 * 1024 || 3 * tile > 200 * 1024)) --sb;
    if (P->N >= 32 && sb >= 2) {
      P->sblk = sb;
      P->Nc = (P->N + sb - 1) / sb;
      unsigned char* dMc = nullptr;
      TRY_ALLOC(dMc, B * (size_t)P->Nc * tile);
      P->dMc = dMc;
    }
  }
  TRY_ALLOC(P->dpsin, B * (P->N + 1) * (size_t)d);
  TRY_ALLOC(P->dchin, B * (P->N + 1) * (size_t)d);
  TRY_ALLOC(P->dphi, B * (P->N + 1) * (size_t)d);
  if (P->direct && !P->ks.large) TRY_ALLOC(P->dnrm, B * (P->N + 1) * 2);
  // checkpoint stride of the literal sub-problem (steps between stored states): by default about the
  // square root of the longest sub-interval, which balances the checkpoints against the segment buffer
  {
    const int nsmax = (P->Nt + P->N - 1) / P->N;   // longest sub-interval of j_n = floor(n Nt / N)
    int S = opt->ckpt_stride > 0 ? opt->ckpt_stride : (int)std::ceil(std::sqrt((double)nsmax));
    P->cks = S < 1 ? 1 : (S > nsmax ? nsmax : S);
    P->nck = (nsmax + P->cks - 1) / P->cks;
  }
  if (P->ks.large) {   // CTA-wide states (bit-flip and Pauli kinds)
    if (P->form == 1 || P->L > 1) {   // ism_iterate runs literal sub-problems
      if ((rc = alloc_literal(P)) != ISM_OK) { free_all(P); delete P; return rc; }
    }
  } else {
    unsigned char* dZ = nullptr;
    TRY_ALLOC(dZ, B * ((size_t)P->Nt + P->N) * P->r2);
    P->dzs = dZ;
    if (P->form == 1 || P->L > 1) {   // ism_iterate runs literal sub-problems
      if ((rc = alloc_literal(P)) != ISM_OK) { free_all(P); delete P; return rc; }
    }
    // first local steps of the assembly path (few problems: latency) by the concurrent sweeps, which
    // store both sub-interval trajectories, while these stay small
    const size_t tb = B * ((size_t)P->Nt + P->N) * GE * P->r2;
    if (!P->direct && P->ks.sweeps2 && P->form == 2 && tb <= kSweeps2MaxBytes) {
      unsigned char* dTb = nullptr;
      TRY_ALLOC(dTb, tb);
      P->dtraj = dTb;
      unsigned char* dT2 = nullptr;
      TRY_ALLOC(dT2, tb);
      P->dtraj2 = dT2;
      P->use_sw2 = true;
    }
  }
  if (P->ks.large) {   // per-slot overlap partials: W warps, or the 2q bit overlaps (Pauli kind)
    unsigned char* dZ = nullptr;
    TRY_ALLOC(dZ, B * ((size_t)P->Nt + P->N) * (P->pauli ? 2 * P->q : P->ks.W) * P->r2);
    P->dzp = dZ;
  }
  if (P->pauli) {
    unsigned char* dC = nullptr;
    TRY_ALLOC(dC, B * (size_t)P->Nt * 2 * P->q * (P->r2 / 2));
    P->dcxy = dC;
    TRY_ALLOC(P->dwts, (size_t)P->m * P->q * 2);
  }
  TRY_ALLOC(P->du, B * P->Nt * P->m);
  TRY_ALLOC(P->duf, B * P->Nt);
  TRY_ALLOC(P->dgrad, B * P->Nt * P->m);
  TRY_ALLOC(P->dJn, B * P->N);
  TRY_ALLOC(P->derr, B * P->N);
  TRY_ALLOC(P->dJ, B);
  TRY_ALLOC(P->dF, B);
  TRY_ALLOC(P->dstatus, 1);
  TRY_ALLOC(P->dcount, 7);
#undef TRY_ALLOC
  if (dry) {
    *bytes_out = P->bytes;
    delete P;
    return ISM_OK;
  }

  cudaError_t e = cudaSuccess;
  auto h2d = [&](void* dst, const void* src, size_t n) {
    if (e == cudaSuccess) e = cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, P->st);
  };
  h2d(P->dH, P->prec == ISM_FP64 ? (const void*)hd.data() : (const void*)hf.data(), hbytes);
  {
    std::vector<double> h0d(d);
    for (int e = 0; e < d; ++e) h0d[e] = p.kind == ISM_H_DENSE ? p.H0[(size_t)e * d + e] : p.H0[e];
    h2d(P->dH0d, h0d.data(), d * sizeof(double));
  }
  h2d(P->djn, jn.data(), jn.size() * sizeof(int));
  {
    std::vector<double> tab(ism::BESSEL_TABLE);
    ism::bessel_table(tab.data());
    h2d(P->dctab, tab.data(), tab.size() * sizeof(double));
  }
  h2d(P->dbeta, beta.data(), beta.size() * sizeof(double));
  h2d(P->dphase, phase.data(), phase.size() * sizeof(double2));
  {
    std::vector<double2> ab(P->N + 1);   // Eq. (cible): a_n = (T - t_n)/T, b_n = t_n/T
    for (int n = 0; n <= P->N; ++n) {
      const double tn = jn[n] * P->tau;
      ab[n] = make_double2((P->T - tn) / P->T, tn / P->T);
    }
    h2d(P->dab, ab.data(), ab.size() * sizeof(double2));
  }
  if (p.alpha) h2d(P->dalpha, p.alpha, P->Nt * sizeof(double));
  if (P->pauli) h2d(P->dwts, p.H1, (size_t)P->m * P->q * 2 * sizeof(double));
  h2d(P->dpsi_i, p.psi_i, 2 * sizeof(double) * d);
  if (p.objective == ISM_OBJ_OVERLAP) h2d(P->dpsi_f, p.psi_f, 2 * sizeof(double) * d);
  else if (e == cudaSuccess) e = cudaMemsetAsync(P->dpsi_f, 0, 2 * sizeof(double) * d, P->st);
  if (p.objective == ISM_OBJ_OBSERVABLE) h2d(P->dO, p.O, sizeof(double) * d * d);
  if (e == cudaSuccess) e = cudaMemsetAsync(P->dstatus, 0, sizeof(int), P->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(P->dcount, 0, 7 * sizeof(unsigned long long), P->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(P->st);   // the host arrays uploaded above are local
  if (e != cudaSuccess) {
    free_all(P);
    delete P;
    return fail(ISM_ECUDA, std::string("plan upload: ") + cudaGetErrorString(e));
  }
  {
    // one ring of as many tile stages as fit in ~200 KB (1..16)
    const size_t tile = (size_t)P->tst * P->r2, budget = 200 * 1024;
    int st = (int)(budget / tile);
    P->chain_stages = st < 1 ? 1 : (st > 16 ? 16 : st);
    P->chain_smem = P->chain_stages * tile;
  }
  *out = P;
  g_err.clear();
  return ISM_OK;
}

}  // namespace

extern "C" {

int ism_plan(const ism_problem* prob, const ism_options* opt, void* cuda_stream, ism_plan_t* out) {
  return plan_build(prob, opt, cuda_stream, out, false, nullptr);
}

int ism_plan_footprint(const ism_problem* prob, const ism_options* opt, size_t* bytes) {
  if (!bytes) return fail(ISM_EINVAL, "null output");
  *bytes = 0;
  int rc = plan_build(prob, opt, nullptr, nullptr, true, bytes);
  if (rc == ISM_OK) g_err.clear();
  return rc;
}

int ism_plan_destroy(ism_plan_t P) {
  if (!P) return ISM_OK;
  cudaSetDevice(P->dev);
  cudaStreamSynchronize(P->st);
  free_all(P);
  delete P;
  return ISM_OK;
}

long long ism_plan_info(ism_plan_t P, int key) {
  if (!P) return -1;
  switch (key) {
    case 0: return P->ks.G;
    case 1: return P->ks.E;
    case 2: return 2 + P->L;
    case 3: return (long long)P->bytes;
    case 4: return (P->gp || P->ks.large || P->direct) ? 0 : (long long)(P->tst * P->r2);
    case 5: return P->ks.large ? 1 : 0;
    case 6: return (P->ks.large || P->direct) ? 2 : 1;
    case 7: return P->Nc ? P->sblk : 1;
    case 8: return P->scheme;
    case 9: return P->wide ? P->ks.GW : (P->direct ? P->ks.G : 0);
    case 10: return P->tc ? 1 : 0;
    case 11: return P->cks;
    default: return -1;
  }
}

int ism_set_profiling(ism_plan_t P, int on) {
  if (!P) return fail(ISM_EINVAL, "null plan");
  P->profiling = on != 0;
  return ISM_OK;
}

int ism_get_stats(ism_plan_t P, ism_stats* out, int reset) {
  if (!P || !out) return fail(ISM_EINVAL, "null argument");
  ISM_CUDA_TRY(cudaSetDevice(P->dev));
  ISM_CUDA_TRY(cudaStreamSynchronize(P->st));
  collect_events(P);
  unsigned long long c[7];   // work counters of two phases, then the norm drift's bits
  ISM_CUDA_TRY(cudaMemcpy(c, P->dcount, sizeof(c), cudaMemcpyDeviceToHost));
  for (int i = 0; i < 3; ++i) { out->ms[i] = P->ms[i]; out->launches[i] = P->launches[i]; }
  out->kernels = P->kernels;
  for (int k = 0; k < 2; ++k) { out->y_apps[k] = c[3 * k]; out->terms[k] = c[3 * k + 1]; out->substeps[k] = c[3 * k + 2]; }
  std::memcpy(&out->norm_drift, &c[6], sizeof(double));
  if (reset) {
    for (int i = 0; i < 3; ++i) { P->ms[i] = 0; P->launches[i] = 0; }
    P->kernels = 0;
    ISM_CUDA_TRY(cudaMemset(P->dcount, 0, sizeof(c)));
  }
  return ISM_OK;
}

int ism_intermediate_states(ism_plan_t P, const double* u, double* phi) {
  if (!P || !u || !phi) return fail(ISM_EINVAL, "null argument");
  int rc = begin(P);
  if (rc) return rc;
  if ((rc = check_device_args(P->dev, {u, phi}))) return rc;
  const double* ud = nullptr;
  if ((rc = stage_in(P, u, (long)P->B * P->Nt * P->m, P->du, &ud, true))) return rc;
  if ((rc = run_states(P, ud, nullptr, 0, 0))) return rc;
  if (P->gp) {
    const size_t blk = 2 * sizeof(double) * (size_t)(P->N + 1) * P->d;   // one set of N+1 states
    ISM_CUDA_TRY(cudaMemcpy2DAsync(phi, 2 * blk, P->dpsin, blk, blk, P->B, cudaMemcpyDefault, P->st));
    ISM_CUDA_TRY(cudaMemcpy2DAsync(reinterpret_cast<char*>(phi) + blk, 2 * blk, P->dchin, blk, blk, P->B,
                                   cudaMemcpyDefault, P->st));
    return finish(P);
  }
  if ((rc = copy_out(P, phi, P->dphi, 2L * P->B * (P->N + 1) * P->d))) return rc;
  return finish(P);
}

int ism_subinterval_grad(ism_plan_t P, const double* phi, const double* u, double* grad, double* Jn) {
  if (!P || !phi || !u || !grad) return fail(ISM_EINVAL, "null argument");
  int rc = begin(P);
  if (rc) return rc;
  if ((rc = check_device_args(P->dev, {phi, u, grad, Jn}))) return rc;
  if (P->tc)
    return fail(ISM_EUNSUPPORTED, "dense d = 128, 256 plans run the two-trajectory form of first local steps only "
                                  "(ism_iterate, ism_gradient); literal sub-problems are not built for them");
  const double* ud = nullptr;
  if ((rc = stage_in(P, u, (long)P->B * P->Nt * P->m, P->du, &ud, true))) return rc;
  if (P->gp) {
    const size_t blk = 2 * sizeof(double) * (size_t)(P->N + 1) * P->d;
    if (!is_device_ptr(phi) && !all_finite(phi, 4L * P->B * (P->N + 1) * P->d))
      return fail(ISM_ENONFINITE, "non-finite value in phi");
    ISM_CUDA_TRY(cudaMemcpy2DAsync(P->dpsin, blk, phi, 2 * blk, blk, P->B, cudaMemcpyDefault, P->st));
    ISM_CUDA_TRY(cudaMemcpy2DAsync(P->dchin, blk, reinterpret_cast<const char*>(phi) + blk, 2 * blk, blk, P->B,
                                   cudaMemcpyDefault, P->st));
    ism::GPParams g = gparams(P, const_cast<double*>(ud));
    g.count = P->dcount + 3;
    ISM_CUDA_TRY(timed(P, 2, 1, [&] { return ism::launch_gp_sub(P->prec, g, P->st); }));
    if ((rc = copy_out(P, grad, P->dgrad, (long)P->B * P->Nt * P->m))) return rc;
    if ((rc = copy_out(P, Jn, P->dJn, (long)P->B * P->N))) return rc;
    return finish(P);
  }
  const long nphi = 2L * P->B * (P->N + 1) * P->d;
  if (is_device_ptr(phi)) {
    ISM_CUDA_TRY(cudaMemcpyAsync(P->dphi, phi, nphi * sizeof(double), cudaMemcpyDeviceToDevice, P->st));
  } else {
    if (!all_finite(phi, nphi)) return fail(ISM_ENONFINITE, "non-finite value in phi");
    ISM_CUDA_TRY(cudaMemcpyAsync(P->dphi, phi, nphi * sizeof(double), cudaMemcpyHostToDevice, P->st));
  }
  if ((rc = alloc_literal(P)) != ISM_OK) return rc;   // first literal use
  ism::KParams k = kparams(P, const_cast<double*>(ud));
  k.update = 0;
  k.count = P->dcount + 3;
  ISM_CUDA_TRY(prep_params(P, k));
  P->kernels += 1;
  ISM_CUDA_TRY(timed(P, 2, 1, [&] { return P->ks.subinterval(k, P->st); }));
  if ((rc = copy_out(P, grad, P->dgrad, (long)P->B * P->Nt * P->m))) return rc;
  if ((rc = copy_out(P, Jn, P->dJn, (long)P->B * P->N))) return rc;
  return finish(P);
}

int ism_iterate(ism_plan_t P, int iters, double* u_inout, double* J_hist, double* err_hist) {
  if (!P || !u_inout) return fail(ISM_EINVAL, "null argument");
  if (iters < 0) return fail(ISM_EINVAL, "iters must be >= 0");
  int rc = begin(P);
  if (rc) return rc;
  if ((rc = check_device_args(P->dev, {u_inout, J_hist, err_hist}))) return rc;
  const long nu = (long)P->B * P->Nt * P->m;
  const bool dev_u = is_device_ptr(u_inout);
  double* ud = nullptr;
  if (dev_u) {
    const double* tmp = nullptr;
    if ((rc = stage_in(P, u_inout, nu, P->du, &tmp, true))) return rc;
    ud = u_inout;
  } else {
    const double* tmp = nullptr;
    if ((rc = stage_in(P, u_inout, nu, P->du, &tmp, true))) return rc;
    ud = P->du;
  }
  const long stride = (long)iters + 1;
  if ((J_hist || err_hist) && (rc = ensure_hist(P, stride))) return rc;
  for (int it = 0; it < iters; ++it) {
    if ((rc = run_states(P, ud, J_hist ? P->dJhist : nullptr, (int)stride, it))) return rc;
    for (int l = 0; l < P->L && P->gp; ++l) {
      ism::GPParams g = gparams(P, ud);
      g.update = 1;
      g.reuse = l == 0;   // phi_n = psi(t_n) at these controls: the forward sweep's stored trajectory
      g.err = l == 0 ? P->derr : nullptr;
      g.Jn = l == 0 ? P->dJn : nullptr;
      g.count = P->dcount + 3;
      ISM_CUDA_TRY(timed(P, 2, 1, [&] { return ism::launch_gp_sub(P->prec, g, P->st); }));
    }
    for (int l = 0; l < P->L && !P->gp; ++l) {
      ism::KParams k = kparams(P, ud);
      k.update = 1;
      k.form = (l == 0 && P->form == 2) ? 1 : 0;
      k.err = l == 0 ? P->derr : nullptr;
      k.Jn = l == 0 ? P->dJn : nullptr;
      k.count = P->dcount + 3;
      if (l > 0) {   // controls moved
        ISM_CUDA_TRY(prep_params(P, k));
        P->kernels += 1;
      }
      if (P->tc) {
        if ((rc = tc_sub(P, k)) != ISM_OK) return rc;
      } else if (k.form && P->use_sw2)
        ISM_CUDA_TRY(timed(P, 2, 2, [&] { return P->ks.sweeps2(k, P->st); }));
      else ISM_CUDA_TRY(timed(P, 2, 1, [&] { return P->ks.subinterval(k, P->st); }));
    }
    if (err_hist) {
      k_err_sum<<<P->B, 32, 0, P->st>>>(P->derr, P->N, P->B, P->derrhist, (int)stride, it);
      P->kernels += 1;
      ISM_CUDA_TRY(cudaGetLastError());
    }
  }
  if (J_hist && (rc = run_states(P, ud, P->dJhist, (int)stride, iters))) return rc;
  if (!dev_u) {   // the updated controls: checked on the device, then copied back
    int blocks = (int)std::min<long>(1024, (nu + 255) / 256);
    if (blocks < 1) blocks = 1;
    ism::k_check_finite<<<blocks, 256, 0, P->st>>>(ud, nu, P->dstatus);
    P->kernels += 1;
    ISM_CUDA_TRY(cudaGetLastError());
    ISM_CUDA_TRY(cudaMemcpyAsync(u_inout, ud, nu * sizeof(double), cudaMemcpyDeviceToHost, P->st));
  }
  // J_hist is [B][iters+1]; err_hist is [B][iters] (packed from the stride-(iters+1) device rows)
  if (J_hist) ISM_CUDA_TRY(cudaMemcpyAsync(J_hist, P->dJhist, (size_t)P->B * stride * sizeof(double), cudaMemcpyDefault, P->st));
  if (err_hist && iters > 0)
    ISM_CUDA_TRY(cudaMemcpy2DAsync(err_hist, iters * sizeof(double), P->derrhist, stride * sizeof(double),
                                   iters * sizeof(double), P->B, cudaMemcpyDefault, P->st));
  if ((rc = finish(P))) return rc;
  return ISM_OK;
}

int ism_gradient(ism_plan_t P, const double* u, double* grad, double* J) {
  if (!P || !u || !grad) return fail(ISM_EINVAL, "null argument");
  int rc = begin(P);
  if (rc) return rc;
  if ((rc = check_device_args(P->dev, {u, grad, J}))) return rc;
  const double* ud = nullptr;
  if ((rc = stage_in(P, u, (long)P->B * P->Nt * P->m, P->du, &ud, true))) return rc;
  if ((rc = run_states(P, ud, nullptr, 0, 0))) return rc;
  if (P->gp) {   // the sub-problem gradients at the adjoint targets are the global gradient
    ism::GPParams g = gparams(P, const_cast<double*>(ud));
    g.update = 0;
    g.reuse = 1;   // psi(t_n) of the sweep just run: its stored trajectory is the sub-problems'
    g.count = P->dcount + 3;
    ISM_CUDA_TRY(timed(P, 2, 1, [&] { return ism::launch_gp_sub(P->prec, g, P->st); }));
  } else {       // Theorem 2 two-trajectory form, scaled by beta_n
    ism::KParams k = kparams(P, const_cast<double*>(ud));
    k.update = 0;
    k.form = 1;
    k.global = 1;
    k.count = P->dcount + 3;
    if (P->tc) {
      if ((rc = tc_sub(P, k)) != ISM_OK) return rc;
    } else if (!P->use_sw2) ISM_CUDA_TRY(timed(P, 2, 1, [&] { return P->ks.subinterval(k, P->st); }));
    else ISM_CUDA_TRY(timed(P, 2, 2, [&] { return P->ks.sweeps2(k, P->st); }));
  }
  if ((rc = copy_out(P, grad, P->dgrad, (long)P->B * P->Nt * P->m))) return rc;
  if ((rc = copy_out(P, J, P->dJ, P->B))) return rc;
  return finish(P);
}

int ism_evaluate(ism_plan_t P, const double* u, double* J, double* F) {
  if (!P || !u) return fail(ISM_EINVAL, "null argument");
  int rc = begin(P);
  if (rc) return rc;
  if ((rc = check_device_args(P->dev, {u, J, F}))) return rc;
  const double* ud = nullptr;
  if ((rc = stage_in(P, u, (long)P->B * P->Nt * P->m, P->du, &ud, true))) return rc;
  if ((rc = run_states(P, ud, nullptr, 0, 0))) return rc;
  if ((rc = copy_out(P, J, P->dJ, P->B))) return rc;
  if ((rc = copy_out(P, F, P->dF, P->B))) return rc;
  return finish(P);
}

}  // extern "C"

// ------------------------------------------------------------------ heterogeneous batch plans
// Rows of different problems that share the kind, d, N and objective run in the same launches (the
// continuous-batching server's shared plans): every row holds its own Hamiltonian, states, step
// count, control time, penalty and step size (ism::RowTab); the direct-sweep kernels, the two-trajectory
// sub-problems and k_phi read them per row.  Mixed precision, the Chebyshev step, one local step; the
// structured kinds (tridiagonal, bit-flip).  A row's results do not depend on the other rows: the
// warp-wide term and step counts only add exact no-ops (zero coefficients, discarded sub-steps,
// inactive steps).
namespace ism {

bool het_batchable(const ism_problem& p, const ism_options& o) {
  if (o.precision != ISM_MIXED || o.scheme != ISM_SCHEME_CHEBYSHEV) return false;
  if (o.local_iters > 1 || o.subproblem_form == 1 || o.step1 == 1 || o.cheb_tol != 0.0) return false;
  if (p.batch > 1 || p.controls > 1) return false;
  if (p.kind == ISM_H_TRIDIAG) return p.d >= 1 && p.d <= 64;
  if (p.kind == ISM_H_BITFLIP) return p.d >= 2 && p.d <= 1024;
  return false;
}

bool het_h1diag(const ism_problem& p) {
  if (p.kind != ISM_H_TRIDIAG) return true;
  for (int e = 0; e < p.d; ++e)
    if (p.H1[e] != 0.0) return true;
  return false;
}

int het_create(int kind, int d, int N, int obj, bool h1diag, int Ntmax, int cap, void* stream, ism_plan_t* out,
               size_t* bytes) {
  ism_plan_s* P = new (std::nothrow) ism_plan_s();
  if (!P) return fail(ISM_ENOMEM, "host allocation");
  P->dry = out == nullptr;
  P->het = true;
  P->d = d; P->kind = kind; P->obj = obj; P->Nt = Ntmax; P->N = N; P->B = cap; P->cap = cap;
  P->prec = ISM_MIXED; P->L = 1; P->form = 2; P->scheme = ISM_SCHEME_CHEBYSHEV;
  P->T = 1.0; P->tau = 1.0 / Ntmax;   // per row in rt
  P->tol = 1e-10;
  P->w = obj == ISM_OBJ_OVERLAP ? 1.0 : 2.0;
  P->max_spin = 1 << 22;
  P->st = reinterpret_cast<cudaStream_t>(stream);
  cudaGetDevice(&P->dev);
  if (!ism::select_kernels(ISM_MIXED, kind, d, &P->ks, h1diag)) {
    delete P;
    return fail(ISM_EUNSUPPORTED, "no compiled kernel for this kind and d");
  }
  P->direct = !P->ks.large;
  P->wide = false;
  P->r2 = sizeof(float2);
  const int GE = P->ks.G * P->ks.E;
  {
    int q = 0;
    while (q < 30 && (1 << q) < d) ++q;
    P->hstride = kind == ISM_H_TRIDIAG ? 4 * d : d + q;
  }
  const size_t B = cap, Ns = (size_t)N, Nts = (size_t)Ntmax;
  int rc = ISM_OK;
  auto fail_out = [&](int code) { free_all(P); delete P; return code; };
#define TRY_HET(ptr, n) if ((rc = dalloc(P, &(ptr), (n))) != ISM_OK) return fail_out(rc);
  unsigned char* dHb = nullptr;
  TRY_HET(dHb, B * P->hstride * sizeof(float));
  P->dH = dHb;
  TRY_HET(P->dH0d, B * d);
  TRY_HET(P->dpsi_i, B * d);
  TRY_HET(P->dpsi_f, B * d);
  if (obj == ISM_OBJ_OBSERVABLE) TRY_HET(P->dO, B * d * d);
  int* jn = nullptr; double* beta = nullptr; double2* phase = nullptr; double2* ab = nullptr;
  double* tau = nullptr; double* bnd = nullptr; double* nrm = nullptr; double* rho = nullptr; double* alpha = nullptr;
  TRY_HET(jn, B * (Ns + 1));
  TRY_HET(beta, B * Ns);
  TRY_HET(phase, B * Ns);
  TRY_HET(ab, B * (Ns + 1));
  TRY_HET(tau, B);
  TRY_HET(bnd, B * 3);
  TRY_HET(nrm, B * 2);
  TRY_HET(rho, B);
  TRY_HET(alpha, B * Nts);
  TRY_HET(P->dcheb, B * Ns * ism::cheb_bytes(ISM_MIXED));
  TRY_HET(P->dpen, B * Ns);
  TRY_HET(P->dctab, (size_t)ism::BESSEL_TABLE);
  TRY_HET(P->dpsin, B * (Ns + 1) * d);
  TRY_HET(P->dchin, B * (Ns + 1) * d);
  TRY_HET(P->dphi, B * (Ns + 1) * d);
  if (P->direct) TRY_HET(P->dnrm, B * (Ns + 1) * 2);
  if (P->ks.large) {
    unsigned char* dZ = nullptr;
    TRY_HET(dZ, B * (Nts + Ns) * P->ks.W * P->r2);
    P->dzp = dZ;
  } else {
    unsigned char* dZ = nullptr;
    TRY_HET(dZ, B * (Nts + Ns) * P->r2);
    P->dzs = dZ;
  }
  TRY_HET(P->du, B * Nts);
  TRY_HET(P->duf, B * Nts);
  TRY_HET(P->dgrad, B * Nts);
  TRY_HET(P->dJn, B * Ns);
  TRY_HET(P->derr, B * Ns);
  TRY_HET(P->dJ, B);
  TRY_HET(P->dF, B);
  TRY_HET(P->dstatus, 1);
  TRY_HET(P->dcount, 7);
#undef TRY_HET
  (void)GE;
  P->rt.jn = jn; P->rt.beta = beta; P->rt.phase = phase; P->rt.ab = ab; P->rt.tau = tau; P->rt.bnd = bnd;
  P->rt.nrm = nrm; P->rt.rho = rho; P->rt.alpha = alpha; P->rt.hstride = P->hstride; P->rt.ustride = Ntmax;
  P->dalpha = alpha;   // penalty sums in k_cheb_prep (rows without a penalty hold zeros)
  if (!out) {
    *bytes = P->bytes;
    delete P;
    return ISM_OK;
  }
  std::vector<double> tab(ism::BESSEL_TABLE);
  ism::bessel_table(tab.data());
  cudaError_t e = cudaMemcpyAsync(P->dctab, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice, P->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(alpha, 0, B * Nts * sizeof(double), P->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(P->du, 0, B * Nts * sizeof(double), P->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(P->dstatus, 0, sizeof(int), P->st);
  if (e == cudaSuccess) e = cudaMemsetAsync(P->dcount, 0, 7 * sizeof(unsigned long long), P->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(P->st);
  if (e != cudaSuccess) return fail_out(fail(ISM_ECUDA, std::string("batch plan upload: ") + cudaGetErrorString(e)));
  *out = P;
  return ISM_OK;
}

int het_set_row(ism_plan_t P, int row, const ism_problem& p, const double* u0, double rho) {
  if (!P || !P->het || row < 0 || row >= P->cap) return fail(ISM_EINVAL, "bad batch row");
  if (p.kind != P->kind || p.d != P->d || p.N != P->N || p.objective != P->obj || p.Nt > P->Nt)
    return fail(ISM_EINVAL, "the problem does not fit this batch plan");
  const int d = p.d, N = p.N;
  std::vector<float> hf = pack_op<float>(p.kind, d, p.H0, p.H1, P->ks.G, P->ks.E);
  hf.resize(P->hstride, 0.f);
  std::vector<double> h0d(d);
  for (int e = 0; e < d; ++e) h0d[e] = p.H0[e];
  Bounds bd = bounds_of(p.kind, d, p.H0, p.H1);
  const double c0 = 0.5 * (bd.lo + bd.hi);
  std::vector<int> jn;
  std::vector<double> beta;
  std::vector<double2> phase;
  ism::partition(p.T, p.Nt, N, c0, &jn, &beta, &phase);
  const double tau = p.T / p.Nt;
  std::vector<double2> ab(N + 1);
  for (int n = 0; n <= N; ++n) {
    const double tn = jn[n] * tau;
    ab[n] = make_double2((p.T - tn) / p.T, tn / p.T);
  }
  const double bnd3[3] = {c0, 0.5 * (bd.hi - bd.lo), bd.h1};
  double nrm2[2] = {0.0, 0.0};
  for (int e = 0; e < d; ++e) {
    nrm2[0] += p.psi_i[2 * e] * p.psi_i[2 * e] + p.psi_i[2 * e + 1] * p.psi_i[2 * e + 1];
    if (p.objective == ISM_OBJ_OVERLAP) nrm2[1] += p.psi_f[2 * e] * p.psi_f[2 * e] + p.psi_f[2 * e + 1] * p.psi_f[2 * e + 1];
  }
  std::vector<double> alpha(P->Nt, 0.0), u(P->Nt, 0.0);
  if (p.alpha) std::copy(p.alpha, p.alpha + p.Nt, alpha.begin());
  if (u0) std::copy(u0, u0 + p.Nt, u.begin());
  cudaError_t e = cudaSuccess;
  auto h2d = [&](void* dst, const void* src, size_t n) {
    if (e == cudaSuccess) e = cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, P->st);
  };
  const size_t r = row;
  h2d(reinterpret_cast<float*>(P->dH) + r * P->hstride, hf.data(), hf.size() * sizeof(float));
  h2d(P->dH0d + r * d, h0d.data(), d * sizeof(double));
  h2d(P->dpsi_i + r * d, p.psi_i, 2 * d * sizeof(double));
  if (p.objective == ISM_OBJ_OVERLAP) h2d(P->dpsi_f + r * d, p.psi_f, 2 * d * sizeof(double));
  else h2d(P->dO + r * d * d, p.O, (size_t)d * d * sizeof(double));
  h2d(const_cast<int*>(P->rt.jn) + r * (N + 1), jn.data(), (N + 1) * sizeof(int));
  h2d(const_cast<double*>(P->rt.beta) + r * N, beta.data(), N * sizeof(double));
  h2d(const_cast<double2*>(P->rt.phase) + r * N, phase.data(), N * sizeof(double2));
  h2d(const_cast<double2*>(P->rt.ab) + r * (N + 1), ab.data(), (N + 1) * sizeof(double2));
  h2d(const_cast<double*>(P->rt.tau) + r, &tau, sizeof(double));
  h2d(const_cast<double*>(P->rt.bnd) + 3 * r, bnd3, 3 * sizeof(double));
  h2d(const_cast<double*>(P->rt.nrm) + 2 * r, nrm2, 2 * sizeof(double));
  h2d(const_cast<double*>(P->rt.rho) + r, &rho, sizeof(double));
  h2d(const_cast<double*>(P->rt.alpha) + r * P->Nt, alpha.data(), P->Nt * sizeof(double));
  if (u0) h2d(P->du + r * P->Nt, u.data(), P->Nt * sizeof(double));
  if (e == cudaSuccess) e = cudaStreamSynchronize(P->st);   // the host vectors above are local
  if (e != cudaSuccess) return fail(ISM_ECUDA, std::string("batch row upload: ") + cudaGetErrorString(e));
  return ISM_OK;
}

int het_move_u(ism_plan_t P, int from, int to) {
  if (from == to) return ISM_OK;
  ISM_CUDA_TRY(cudaMemcpyAsync(P->du + (size_t)to * P->Nt, P->du + (size_t)from * P->Nt, P->Nt * sizeof(double),
                               cudaMemcpyDeviceToDevice, P->st));
  return ISM_OK;
}

int het_set_rho(ism_plan_t P, int row, double rho) {
  ISM_CUDA_TRY(cudaMemcpyAsync(const_cast<double*>(P->rt.rho) + row, &rho, sizeof(double), cudaMemcpyHostToDevice, P->st));
  ISM_CUDA_TRY(cudaStreamSynchronize(P->st));
  return ISM_OK;
}

// One pass of Algorithm 1 (a)-(d) on rows [0, rows): J at the rows' current controls into J (host),
// the controls updated in place with each row's step size (0: the row is only evaluated).
int het_step(ism_plan_t P, int rows, double* J) {
  if (!P || !P->het || rows < 1 || rows > P->cap) return fail(ISM_EINVAL, "bad batch rows");
  P->B = rows;
  int rc = begin(P);
  if (rc) return rc;
  if ((rc = run_states(P, P->du, nullptr, 0, 0))) return rc;
  ism::KParams k = kparams(P, P->du);
  k.update = 1;
  k.form = 1;
  k.err = P->derr;
  k.Jn = P->dJn;
  k.count = P->dcount + 3;
  ISM_CUDA_TRY(timed(P, 2, 1, [&] { return P->ks.subinterval(k, P->st); }));
  ISM_CUDA_TRY(cudaMemcpyAsync(J, P->dJ, rows * sizeof(double), cudaMemcpyDeviceToHost, P->st));
  return finish(P);
}

int het_get_u(ism_plan_t P, int row, double* u, int Nt) {
  ISM_CUDA_TRY(cudaMemcpyAsync(u, P->du + (size_t)row * P->Nt, Nt * sizeof(double), cudaMemcpyDeviceToHost, P->st));
  ISM_CUDA_TRY(cudaStreamSynchronize(P->st));
  return ISM_OK;
}

long long het_kernels(ism_plan_t P) { return P ? P->kernels : 0; }

}  // namespace ism
