// ism_launch.h -- host-side table of the compiled kernel variants (one translation unit per
// Hamiltonian structure, instantiated for FP32 and FP64 and for each supported dimension class).
#pragma once
#include <cuda_runtime.h>

namespace ism {

struct KParams;
struct ChainParams;

// Raise a kernel's dynamic shared-memory cap, once per kernel and device, to all the device allows
// beside the kernel's static shared memory.  Launches then pass their own (smaller) sizes; plans on
// other host threads (the serving loop) cannot lower the cap under a launch in flight, which a
// per-launch cudaFuncSetAttribute with differing sizes would.
cudaError_t raise_smem_cap(const void* kernel);

typedef cudaError_t (*LaunchFn)(const KParams&, cudaStream_t);

struct KernelSet {
  LaunchFn assemble = nullptr;
  LaunchFn subinterval = nullptr;
  LaunchFn sweeps2 = nullptr;     // concurrent two-trajectory sweeps + gradient pass
  LaunchFn gsweep = nullptr;      // direct global sweeps (Algorithm 1 (a)-(b) without assembly)
  // the same sweeps in the assembly's lane layout (fewer lanes, more elements per lane): fewer
  // shuffles per element, for batches that give every SM two CTAs of it (FP32 packed path only)
  LaunchFn gsweep_wide = nullptr;
  int GW = 0;                     // lanes per state of gsweep_wide
  LaunchFn prep = nullptr;        // per-sub-interval parameters, when not k_cheb_prep (several controls)
  int G = 0, E = 0;          // lanes per state, elements per lane (sub-interval sweep)
  int GA = 0;                // lanes per state in the assembly
  size_t op_smem = 0;        // dynamic shared memory of the op (dense H pairs)
  // large d (one state per CTA): direct global sweeps instead of assembly + chain
  bool large = false;
  LaunchFn lsweep = nullptr;
  int W = 0;                 // warps per state
};

// prec: 0 = FP64, 1 = FP32 propagation.  Return false when d is outside the compiled range.
bool kernels_tridiag(int prec, int d, bool h1diag, KernelSet* ks);   // h1diag: H1 has a diagonal
bool kernels_bitflip(int prec, int d, KernelSet* ks);
bool kernels_dense(int prec, int d, KernelSet* ks);
bool kernels_dense_cx(int prec, int d, KernelSet* ks);   // complex Hermitian H0, H1
bool kernels_large_bitflip(int prec, int d, KernelSet* ks);   // d = 128, 256, 512, 1024
bool kernels_pauli(int prec, int d, KernelSet* ks);   // several controls, Pauli structure, d = 128..1024
// Crank-Nicolson step (FP64 or FP32 propagation): tridiagonal, bit-flip (d <= 64) and dense kinds
bool kernels_cn(int prec, int kind, int d, bool h1diag, KernelSet* ks);
cudaError_t launch_chain(int prec, const ChainParams& p, size_t smem, cudaStream_t st);   // k_chain + k_phi
cudaError_t launch_phi(int prec, const ChainParams& p, cudaStream_t st);                   // k_phi alone
bool select_kernels(int prec, int kind, int d, KernelSet* ks, bool h1diag = true, bool cx = false);
// per-sub-interval propagator parameters (one warp each) from the current controls
cudaError_t launch_cheb_prep(int prec, const KParams& p, cudaStream_t st);
size_t cheb_bytes(int prec);
// 1/(m! (m+k)!) for k < 32, m <= 24, row-major (k, m): the Bessel series table of the parameters
void bessel_table(double* out);
constexpr int BESSEL_TABLE = 32 * 25;

}  // namespace ism

#include <vector>
#include "ism.h"

namespace ism {

// Host helpers shared by the entry points (defined in ism_api.cu).
struct Bounds { double lo, hi, h1; };
// H0i, H1i: imaginary parts of a complex Hermitian dense H (or null)
Bounds bounds_of(int kind, int d, const double* H0, const double* H1, const double* H0i = nullptr,
                 const double* H1i = nullptr);
template <typename R>
std::vector<R> pack_op(int kind, int d, const double* H0, const double* H1, int G, int E, const double* H0i = nullptr,
                       const double* H1i = nullptr);
int validate_problem(const ism_problem& p, int precision);
// The partition of Sec. 2 and its per-sub-interval weights, computed in one place so that every
// entry point uploads the same bits: j_n = floor(n Nt / N) (N+1 values), beta_n = T / (t_{n+1} - t_n)
// with t_n = j_n tau (N values), and (cos, sin) of the segment phase c0 tau (j_{n+1} - j_n) (N values).
void partition(double T, int Nt, int N, double c0, std::vector<int>* jn, std::vector<double>* beta,
               std::vector<double2>* phase);

// Heterogeneous batch plans (ism_api.cu): rows of different problems sharing kind, d, N and objective,
// used by the serving loop to run requests in shared launches.  het_create with out == NULL only
// sizes the plan (*bytes).  het_step runs one ISM pass on rows [0, rows) and returns J at the rows'
// controls before the pass; a row with step size 0 is evaluated only.
bool het_batchable(const ism_problem& p, const ism_options& o);
bool het_h1diag(const ism_problem& p);
int het_create(int kind, int d, int N, int obj, bool h1diag, int Ntmax, int cap, void* stream, ism_plan_t* out,
               size_t* bytes);
int het_set_row(ism_plan_t P, int row, const ism_problem& p, const double* u0, double rho);
int het_move_u(ism_plan_t P, int from, int to);
int het_set_rho(ism_plan_t P, int row, double rho);
int het_step(ism_plan_t P, int rows, double* J);
int het_get_u(ism_plan_t P, int row, double* u, int Nt);
long long het_kernels(ism_plan_t P);
int set_error(int code, const char* msg);
void clear_error();

}  // namespace ism
