// ism_gp.h -- parameters and launchers of the Gross-Pitaevskii kernels (ism_gp.cu).
#pragma once
#include <cuda_runtime.h>

namespace ism {

struct GPParams {
  int n, Nt, N, B;
  double tau, T, L, xmin, dx, g, rho;
  int pot;                // 0: V = (x - u)^2/2; 1: the double well of separation dw
  double dw;
  const int* jn;          // [N+1]
  double* u;              // [B][Nt]
  const double2* psi_i;   // [n]
  const double2* psi_f;   // [n]
  void* traj;             // cks == 0: [B][Nt+1][n] complex R: a_j = K psi_j
  int cks, nck;           // checkpoint stride (0: the whole trajectory in traj) and checkpoints per sub-interval
  void* gck;              // cks > 0: [B][N][nck][n] a_j at j = j_n + k cks
  void* segb;             // cks > 0: [B][N][cks][n] one recomputed segment per (problem, sub-interval)
  double2* psin;          // [B][N+1][n] psi(t_n)
  double2* chin;          // [B][N+1][n] chi(t_n) = lambda_{j_n}
  double* grad;           // [B][Nt]
  double* Jn;             // [B][N]
  double* err;            // [B][N]
  double* J;              // [B]
  double* F;              // [B]
  double* Jhist;          // [B][hist_stride] or null
  int hist_stride, hist_k;
  int* status;
  unsigned long long* count;   // [2]: FFT pairs (sequential sweeps), FFT pairs (sub-interval sweeps)
  int update;
  int reuse;              // k_gp_sub: the sub-problems start from psi(t_n) at the controls of the last
                          // k_gp_forward (a first local step), so their forward trajectories are its
                          // stored states (traj, or the checkpoints gck): only the adjoint runs
  const void* tab;        // [7n] complex R: the plan's twiddle, kinetic-factor and grid tables (k_gp_tables)
};

// prec: 0 FP64, 1 FP32.  n must be 64 or 512 (radix-8 Stockham; the states in shared memory, the
// per-plan tables in global memory, filled once by launch_gp_tables before the first sweep).
bool gp_supported(int n);
size_t gp_table_bytes(int prec, int n);
cudaError_t launch_gp_tables(int prec, const GPParams& p, cudaStream_t st);   // fills p.tab (once per plan)
cudaError_t launch_gp_forward(int prec, const GPParams& p, cudaStream_t st);
cudaError_t launch_gp_adjoint(int prec, const GPParams& p, cudaStream_t st);
cudaError_t launch_gp_sub(int prec, const GPParams& p, cudaStream_t st);

}  // namespace ism
