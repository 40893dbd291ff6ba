// ism_tc.h -- dense Hamiltonians of dimension d = 128 or 256 propagated on the tensor cores
// (ism_tc.cu): parameters and launchers.
#pragma once
#include <cuda_runtime.h>

namespace ism {

// One complex state carried by the stacked sweep (two real columns of the state matrix).
struct TcItem {
  int b;      // problem; -1: padding (the state stays zero, nothing is stored)
  int n;      // global sweep: unused; sub-interval sweep: the sub-interval
  int role;   // sub-interval sweep: 0 psi (from psi(t_n)), 1 chi (from chi(t_n)); pairs (2q, 2q+1)
  int dir;    // global sweep: 0 psi forward in time (U), 1 chi backward (U^H)
};

struct TcParams {
  int d, Nt, N, B, obj;
  int mode;                // 0: global sweeps (Algorithm 1 (a)-(b)); 1: sub-interval sweeps (step (c))
  int nitems;              // items of the launch (a multiple of the items per CTA)
  int nsteps;              // steps every item runs (sub-interval sweeps: the longest sub-interval)
  const TcItem* items;
  const int* jn;           // [N+1]
  const float* uf;         // [B][Nt] FP32 controls (written by k_cheb_prep)
  const void* cheb;        // [B][N] Cheb<float>: the propagator parameters of each sub-interval
  const double2* psi_i;    // [d]
  const double2* psi_f;    // [d]
  double2* psin;           // [B][N+1][d] psi(t_n)
  double2* chin;           // [B][N+1][d] chi(t_n)
  float2* zs;              // sub-interval sweeps: [B][Nt+N] overlaps <chi_s|H1 psi_s>
  float* vstate;           // [CTAs][2][columns][d] FP32 states (hi, lo) of each CTA's columns
  int* status;
  int max_spin;
  unsigned long long* count;   // [3]: applications of Y, accumulated terms, exp sub-steps (or null)
};

// Tensor maps of the TF32 hi and lo parts of [H0; H1] (2d rows of d floats each).
struct TcMaps {
  alignas(64) unsigned char hi[128];
  alignas(64) unsigned char lo[128];
};

bool tc_supported(int d);
int tc_items_per_cta(int d);
size_t tc_smem_bytes(int d);
// Encode the tensor maps over device arrays hi, lo ([2d][d] floats each).
cudaError_t tc_encode_maps(TcMaps* m, const float* hi, const float* lo, int d);
cudaError_t launch_tc_sweep(const TcMaps& m, const TcParams& p, cudaStream_t st);
struct KParams;
// gradient, J_n, Err and ascent of every (problem, n) from the stored overlaps (two-trajectory form)
cudaError_t launch_tc_zgrad(const KParams& p, cudaStream_t st);
// chi(T) = O psi(T) in FP64 for the observable objective, before the backward global sweep
cudaError_t launch_tc_chiT(const double* O, double2* psin, double2* chin, int d, int N, int B, cudaStream_t st);

}  // namespace ism
