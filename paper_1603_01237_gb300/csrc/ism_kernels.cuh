// ism_kernels.cuh -- the ISM hot-path kernels, templated on precision R and Hamiltonian structure Op.
//
//   k_assemble    Sec. 3 propagator assembly: M_n = prod_{j in sub-interval n} U_j, one group per
//                 (problem, n, column); the column e_k is propagated through the sub-interval.
//   k_chain       Algorithm 1 steps (a)-(b): psi(t_{n+1}) = M_n psi(t_n), chi(t_n) = M_n^H chi(t_{n+1}),
//                 phi_n = a_n psi(t_n) + b_n chi(t_n) (Eq. (cible), FP64), J and F at u.  One CTA per
//                 problem; M_{n+1} is prefetched into shared memory by a TMA bulk copy while M_n is used.
//   k_subinterval Algorithm 1 step (c): per (problem, n) the forward state psi_n from phi_n
//                 (Eq. (dirpara)), then the backward adjoint and the per-step gradient of J_n
//                 (proof of Theorem 2), and optionally the ascent step of Eq. (gradStep).
#pragma once
#include <type_traits>

#include "ism_device.cuh"

namespace ism {

// Per-problem data of a heterogeneous batch: problems that share the kind, d, N, precision and
// objective but each have their own Hamiltonian, initial and target states, step count, control time,
// penalty and step size (the continuous-batching server merges such requests into one plan).  When
// KParams::het is set, the direct-sweep kernels read these instead of the plan-wide fields.
struct RowTab {
  const int* jn;          // [B][N+1] step boundaries
  const double* beta;     // [B][N]
  const double2* phase;   // [B][N] (cos, sin) of each segment's global phase
  const double2* ab;      // [B][N+1] (a_n, b_n) of Eq. (cible)
  const double* tau;      // [B]
  const double* bnd;      // [B][3] spectral centre c0, half-width r0 and the |H1| bound
  const double* nrm;      // [B][2] |psi_i|^2, |psi_f|^2
  const double* rho;      // [B] ascent step (0: the problem takes no step)
  const double* alpha;    // [B][ustride] penalty weights, or null
  long hstride;           // elements of one problem's packed op data
  long ustride;           // row stride of u, uf, grad and alpha (the longest Nt)
};

// The plan-wide or the per-problem view of problem b's data.
struct RowView {
  const int* jn;
  const double* beta;
  const double2* phase;
  const double* alpha;
  double tau, c0, r0, h1n, rho;
  long us;                // row stride of u, uf, grad
  long hoff, doff;        // offsets of b's op data (elements) and of its d-vectors (psi_i, psi_f, H0d)
};

struct KParams {
  int d, Nt, N, B, ldm, dpad;
  double tau, T, c0, r0, h1n, tol, rho, w;
  const int* jn;          // [N+1] step boundaries
  const double* beta;     // [N]
  const double* alpha;    // [Nt] or null
  const void* H;          // packed op data (element type R)
  const double* H0d;      // FP64 diagonal of H0 (tridiagonal and bit-flip kinds)
  const void* cheb;       // [B][N] Cheb<R>: propagator parameters per sub-interval (k_cheb_prep)
  double* pen;            // [B][N] sum_j alpha_j u_j^2 per sub-interval (k_cheb_prep), or null
  const double* ctab;     // Bessel series table for k_cheb_prep
  const double2* phase;   // [N] (cos, sin) of c0 tau (j_{n+1} - j_n), the segment phases
  double* u;              // [B][Nt]
  const double2* phi;     // [B][N+1][d]
  void* M;                // [B][N] tiles of tile_stride R2: [d cols][ldm rows], ldm odd >= d
  long tile_stride;
  void* traj;             // [B][Nt+N][G*E] (R2)  H1 psi_n(t_j) per step
  void* traj2;            // [B][Nt+N][G*E] (R2)  chi^ per step (concurrent two-trajectory sweeps)
  void* zs;               // [B][Nt+N] (R2)  per-step overlap z_s of the sub-interval sweeps
  void* ckpt;             // [B][N][nck][hi (, lo)][G*E] (R2)  checkpoints of the literal sub-problem
  void* segb;             // [B][N][cks][G*E] (R2)  H1 psi_n of the segment being stepped back
  int cks, nck;           // checkpoint stride (steps) and checkpoints per sub-interval
  double* grad;           // [B][Nt]
  double* Jn;             // [B][N]
  double* err;            // [B][N]
  int* status;
  unsigned long long* count;   // [3]: Y applications, accumulated terms, exp sub-steps (or null)
  const double2* psin;         // [B][N+1][d] psi(t_n) (form 1)
  const double2* chin;         // [B][N+1][d] chi(t_n) (form 1)
  int form;                    // 0: literal sub-problem from phi; 1: Theorem 2 two-trajectory form
  int global;                  // form 1 only: scale the gradient to the full objective (beta_n g_n)
  int update;
  int max_spin;
  float* uf;                   // [B][Nt] FP32 copy of u (written by k_cheb_prep)
  int scheme;                  // 0: Chebyshev series; 1: Crank-Nicolson (r0, h1n: off-diagonal row-sum
                               //    bounds of H0 and H1)
  // several controls (Pauli structure): u and grad are [B][Nt][m]
  int m, q;
  const double* wts;           // [m][q][2] weights (ax, ay) of X_b, Y_b in control c
  void* cxy;                   // [B][Nt][2q] (R) step coefficients cx_b, cy_b (k_pauli_prep)
  void* zq;                    // [B][Nt+N][2q] (R2) per-slot overlaps <delta|X_b psi>, <delta|Y_b psi>
  double* nrm_w;               // [B][N+1][2] |psi(t_n)|^2, |chi(t_n)|^2 from k_gsweep (FP64), or null
  // direct global sweeps (large d): inputs and FP64 outputs, per-warp overlap partials
  const double2* psi_i;        // [d]
  const double2* psi_f;        // [d]
  const double* O;             // [d][d] (observable objective)
  int obj;
  double2* psin_w;             // [B][N+1][d] psi(t_n)
  double2* chin_w;             // [B][N+1][d] chi(t_n)
  void* zp;                    // [B][Nt+N][W] (R2)
  int het;                     // heterogeneous batch: problem data from rt
  RowTab rt;
};

template <bool HET>
__device__ __forceinline__ RowView row_view(const KParams& p, int b) {
  RowView r;
  if constexpr (HET) {
    r.jn = p.rt.jn + (long)b * (p.N + 1);
    r.beta = p.rt.beta + (long)b * p.N;
    r.phase = p.rt.phase + (long)b * p.N;
    r.alpha = p.rt.alpha ? p.rt.alpha + (long)b * p.rt.ustride : nullptr;
    r.tau = p.rt.tau[b];
    r.c0 = p.rt.bnd[3 * b];
    r.r0 = p.rt.bnd[3 * b + 1];
    r.h1n = p.rt.bnd[3 * b + 2];
    r.rho = p.rt.rho[b];
    r.us = p.rt.ustride;
    r.hoff = (long)b * p.rt.hstride;
    r.doff = (long)b * p.d;
  } else {
    r.jn = p.jn; r.beta = p.beta; r.phase = p.phase; r.alpha = p.alpha;
    r.tau = p.tau; r.c0 = p.c0; r.r0 = p.r0; r.h1n = p.h1n; r.rho = p.rho;
    r.us = p.Nt; r.hoff = 0; r.doff = 0;
  }
  return r;
}

struct ChainParams {
  int d, Nt, N, B, ldm, obj;
  double tau, T;
  const void* M;          // as KParams::M
  const double2* psi_i;   // [d]
  const double2* psi_f;   // [d]
  const double* O;        // [d][d]
  const double* alpha;    // [Nt] or null
  const double* u;        // [B][Nt]
  const int* jn;
  const double2* ab;      // [N+1] (a_n, b_n) of Eq. (cible), computed on the host in FP64
  double2* psin;          // [B][N+1][d]
  double2* chin;          // [B][N+1][d]
  void* stage;            // [B][2][N+1][d] R2: chain results before the FP64 conversion in k_phi
  const double* pen;      // [B][N] penalty sums per sub-interval (from k_cheb_prep), or null
  double2* phi;           // [B][N+1][d]
  double* J;              // [B]
  double* F;              // [B]
  double* Jhist;          // [B][hist_stride] or null
  int hist_stride, hist_k;
  int stages;             // bulk-copy ring depth per chain (2..CHAIN_MAX_STAGES)
  long tile_stride;       // R2 elements between consecutive tiles (d*ldm rounded up to even)
  int* status;
  int max_spin;
  int src64;              // k_phi: psi(t_n), chi(t_n) are already FP64 in psin, chin (direct sweeps)
  // blocked chain: Nc coarse steps over the products of sblk consecutive tiles (0: plain chain)
  void* Mc;               // [B][Nc] tiles: P_k = M_{k sblk + len_k - 1} ... M_{k sblk}
  int Nc, sblk;
  unsigned long long* drift;   // largest relative norm drift seen by k_phi (double bits), or null
  double nrm_psi_i, inv_nrm_psi_i;   // |psi_i|^2 and its inverse
  double nrm_chi_T;                  // |psi_f|^2 (overlap objective), or -1: summed per problem
  const double* nrm;                 // [B][N+1][2] squared norms from the direct sweeps, or null
  int het;                           // heterogeneous batch: psi_i, (a_n, b_n), tau and the reference
  RowTab rt;                         //   norms per problem (k_phi)
};

template <typename R> __device__ __forceinline__ R ldu_ro(const double* u, long i) { return (R)__ldg(u + i); }
template <typename R> __device__ __forceinline__ R ldu(const double* u, long i) { return (R)u[i]; }
// A control in the propagation precision: FP32 sweeps read the FP32 copy that k_cheb_prep writes
// (a conversion from FP64 would run on the FP64 pipe at every step).
template <typename R> __device__ __forceinline__ R uval(const double* u, const float* uf, long i) {
  if constexpr (sizeof(R) == 4) return __ldg(uf + i);
  else return __ldg(u + i);
}

// Work accounting: one group adds its applications of Y, accumulated series terms and exp sub-steps.
template <typename R>
__device__ __forceinline__ void count_work(unsigned long long* c, const Cheb<R>& ch, long steps, int lg) {
  if (c && lg == 0 && steps > 0) {
    atomicAdd(c + 0, (unsigned long long)(steps * ch.S * (ch.K - 1)));
    atomicAdd(c + 1, (unsigned long long)(steps * ch.S * ch.K));
    atomicAdd(c + 2, (unsigned long long)(steps * ch.S));
  }
}

// ST_NONFINITE when any of x[0..n) is NaN or infinite (a template so that every translation unit
// that includes this header may launch it).
template <int = 0>
__global__ void k_check_finite(const double* x, long n, int* status) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    if (!isfinite(x[i])) { atomicOr(status, ST_NONFINITE); return; }
}

// ------------------------------------------------------------------------------ k_assemble
template <typename R, class Op>
__global__ void __launch_bounds__(128, Op::ASM_MINB) k_assemble(KParams p) {
  constexpr int G = Op::G, E = Op::E, GPB = 128 / G;
  constexpr bool COMP = sizeof(R) == 4;
  using R2 = typename C2<R>::T;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ Cheb<R> chs[GPB];
  const int lg = threadIdx.x % G, gib = threadIdx.x / G;
  const long gid = (long)blockIdx.x * GPB + gib;
  const long total = (long)p.B * p.N * p.dpad;   // multiple of 32/G, so validity is warp-uniform
  if (Op::G * Op::E == Op::DP_SMEM) {            // dense: stage H pairs for the whole CTA
    const R* src = reinterpret_cast<const R*>(p.H);
    R* dst = reinterpret_cast<R*>(smem_raw);
    for (int i = threadIdx.x; i < Op::SMEM_WORDS; i += blockDim.x) dst[i] = src[i];
    __syncthreads();
  }
  if (gid >= total) return;
  const int col = (int)(gid % p.dpad);
  const long bn = gid / p.dpad;
  const int n = (int)(bn % p.N), b = (int)(bn / p.N);
  const int j0 = p.jn[n], j1 = p.jn[n + 1];
  const double* ub = p.u + (long)b * p.Nt;
  const float* ufb = p.uf + (long)b * p.Nt;

  Cheb<R>& ch = chs[gib];
  int Kw, Sw;
  cheb_load<G, R>(ch, reinterpret_cast<const Cheb<R>*>(p.cheb) + bn, lg, Kw, Sw);

  Op op;
  op.load(reinterpret_cast<const R*>(p.H), p.H0d, p.d, lg, smem_raw);
  op.scale(p.H0d, p.d, lg, ch);
  Vec<R, E> v, lo;
  if constexpr (sizeof(R) == 4 && Op::PACKED) {   // packed FP32: both halves per instruction
    VecP<E> pv, pl;
#pragma unroll
    for (int r = 0; r < E; ++r) {
      pv.z[r] = make_float2((lg * E + r == col) ? 1.f : 0.f, 0.f);
      pl.z[r] = make_float2(0.f, 0.f);
    }
    float ua = __ldg(ufb + (j0)), ub1 = j0 + 1 < j1 ? __ldg(ufb + (j0 + 1)) : 0.f;
    for (int j = j0; j < j1; ++j) {
      const float uj = ua;
      ua = ub1;
      if (j + 2 < j1) ub1 = __ldg(ufb + (j + 2));
      op.set_u(uj, ch, lg);
      cheb_step_p<false, true>(pv, pl, op, ch, Kw, Sw);
    }
#pragma unroll
    for (int r = 0; r < E; ++r) {
      v.re[r] = pv.z[r].x; v.im[r] = pv.z[r].y;
      lo.re[r] = pl.z[r].x; lo.im[r] = pl.z[r].y;
    }
  } else {
#pragma unroll
    for (int r = 0; r < E; ++r) {
      v.re[r] = (lg * E + r == col) ? R(1) : R(0);
      v.im[r] = R(0);
      lo.re[r] = R(0);
      lo.im[r] = R(0);
    }

    // controls two steps ahead in registers
    R ua = uval<R>(ub, ufb, j0), ub1 = j0 + 1 < j1 ? uval<R>(ub, ufb, j0 + 1) : R(0);
    for (int j = j0; j < j1; ++j) {
      const R uj = ua;
      ua = ub1;
      if (j + 2 < j1) ub1 = uval<R>(ub, ufb, j + 2);
      op.set_u(uj, ch, lg);
      prop_step<false, COMP>(v, lo, op, ch, Kw, Sw);
    }
  }
  if (col < p.d) {
    count_work<R>(p.count, ch, j1 - j0, lg);
    const double sn = ch.sph, cs = ch.cph;   // global phase exp(-i c (t_{n+1} - t_n)) of the sub-interval
    R2* M = reinterpret_cast<R2*>(p.M) + bn * p.tile_stride + (long)col * p.ldm;
#pragma unroll
    for (int r = 0; r < E; ++r) {
      int e = lg * E + r;
      if (e < p.d) {
        double yr, yi;
        phase_rotate(cs, sn, false, (double)v.re[r] + (double)lo.re[r], (double)v.im[r] + (double)lo.im[r], yr, yi);
        R2 z; z.x = (R)yr; z.y = (R)yi; M[e] = z;
      }
    }
  }
}

// ------------------------------------------------------------------------- sub-problem helpers
// Per-step overlap slots: z_s = <a_s|H1 b_s> of step s of sub-interval n at zs[b][j_n + n + s],
// s = 0..ns (one complex number per step; the trailing slot of each sub-interval holds its end point).
//
// FP64 pass over the steps, lanes of the group on different steps: the trapezoid gradient term of
// step j from the slots s, s+1 (Crank-Nicolson: slot s holds both ends), the penalty, Err and the
// ascent step; J_n = w(-|delta(t_{n+1})|^2/2) - penalty.
template <int G, bool CNs, bool HET, typename R2>
__device__ __forceinline__ void sub_grad_pass(const KParams& p, const R2* zs, int b, int n, long gid, int j0, int ns,
                                              double cPhi, double sPhi, double nrm, int lg, int stride, bool valid) {
  const RowView rv = row_view<HET>(p, b);   // formed here, not kept live across the caller's sweep
  const double beta = rv.beta[n];
  const double ht = 0.5 * rv.tau * p.w / ((p.form && !p.global) ? beta : 1.0);
  const double tb = rv.tau / (p.global ? 1.0 : beta);   // Theorem 2: beta_n g_n is the gradient of J
  const double step = rv.rho * beta / rv.tau;
  double* ub = p.u + (long)b * rv.us;
  double* gb = p.grad + (long)b * rv.us;
  double err = 0.0, pen = 0.0;
  for (int s = lg; s < ns; s += stride) {
    const int j = j0 + s;
    const double uj = ub[j];
    const double al = rv.alpha ? rv.alpha[j] : 0.0;
    const R2 za = zs[s], zb = zs[s + 1];
    // Im(exp(-i Phi) z) for the two ends of step j
    const double Ia = cPhi * (double)za.y - sPhi * (double)za.x;
    const double Ib = CNs ? 0.0 : cPhi * (double)zb.y - sPhi * (double)zb.x;
    const double g = ht * (Ia + Ib) - tb * al * uj;
    err += fabs(g);
    pen += al * uj * uj;
    if (valid) {
      gb[j] = g;
      if (p.update) ub[j] = uj + step * g;
    }
  }
  err = g_sum<G>(err);
  pen = g_sum<G>(pen);
  if (lg == 0 && valid) {
    if (p.Jn) p.Jn[gid] = p.w * (-0.5 * nrm) - 0.5 * tb * pen;
    if (p.err) p.err[gid] = err;
  }
}

// z = <a|h> over the group, products in the propagation precision
template <int G, typename R, int E>
__device__ __forceinline__ void g_zdot(const Vec<R, E>& a, const Vec<R, E>& h, R& zr, R& zi) {
  R xr = R(0), xi = R(0);
#pragma unroll
  for (int r = 0; r < E; ++r) {
    xr = fma(a.re[r], h.re[r], fma(a.im[r], h.im[r], xr));
    xi = fma(a.re[r], h.im[r], fma(-a.im[r], h.re[r], xi));
  }
  zr = g_sum<G>(xr);
  zi = g_sum<G>(xi);
}
// the same on packed FP32 states: (re re, im im) and (re im, -im re) pair sums
template <int G, int E>
__device__ __forceinline__ void g_zdot_p(const VecP<E>& a, const VecP<E>& h, float& zr, float& zi) {
  float2 s1 = make_float2(0.f, 0.f), s2 = make_float2(0.f, 0.f);
#pragma unroll
  for (int r = 0; r < E; ++r) {
    s1 = fma2(a.z[r], h.z[r], s1);
    s2 = fma2(a.z[r], make_float2(h.z[r].y, -h.z[r].x), s2);
  }
  zr = g_sum<G>(s1.x + s1.y);
  zi = g_sum<G>(s2.x + s2.y);
}

// A group's share of an FP64 state (d elements, zero padded) as hi (+ lo for FP32 propagation).
template <typename R, int E>
__device__ __forceinline__ void load_group_state(Vec<R, E>& v, Vec<R, E>& lo, const double2* src, int d, int lg) {
#pragma unroll
  for (int r = 0; r < E; ++r) {
    const int e = lg * E + r;
    const double2 z = e < d ? src[e] : make_double2(0.0, 0.0);
    v.re[r] = (R)z.x;
    v.im[r] = (R)z.y;
    lo.re[r] = sizeof(R) == 4 ? (R)(z.x - (double)v.re[r]) : R(0);
    lo.im[r] = sizeof(R) == 4 ? (R)(z.y - (double)v.im[r]) : R(0);
  }
}
template <typename R, int E>
__device__ __forceinline__ void to_packed(const Vec<R, E>& v, const Vec<R, E>& lo, VecP<E>& pv, VecP<E>& pl) {
#pragma unroll
  for (int r = 0; r < E; ++r) {
    pv.z[r] = make_float2((float)v.re[r], (float)v.im[r]);
    pl.z[r] = make_float2((float)lo.re[r], (float)lo.im[r]);
  }
}

// Preamble shared by the sub-interval kernels: group coordinates, the dense op's shared-memory copy.
#define ISM_SUB_PREAMBLE                                                                              \
  constexpr int G = Op::G, E = Op::E, GPB = 128 / G, GE = G * E;                                      \
  constexpr bool COMP = sizeof(R) == 4;                                                               \
  constexpr bool PK = COMP && Op::PACKED;                                                             \
  using R2 = typename C2<R>::T;                                                                       \
  extern __shared__ __align__(128) unsigned char smem_raw[];                                          \
  __shared__ Cheb<R> chs[GPB];                                                                        \
  const int lg = threadIdx.x % G, gib = threadIdx.x / G;                                              \
  const long gid0 = (long)blockIdx.x * GPB + gib;                                                     \
  const long total = (long)p.B * p.N;                                                                 \
  if (Op::G * Op::E == Op::DP_SMEM) {                                                                 \
    const R* src_ = reinterpret_cast<const R*>(p.H);                                                  \
    R* dst_ = reinterpret_cast<R*>(smem_raw);                                                         \
    for (int i = threadIdx.x; i < Op::SMEM_WORDS; i += blockDim.x) dst_[i] = src_[i];  \
    __syncthreads();                                                                                  \
  }                                                                                                   \
  /* warps whose groups are all past the end leave; partially valid warps keep every lane running */ \
  const long warp_first = ((long)blockIdx.x * GPB + (threadIdx.x / 32) * (32 / G));                   \
  if (warp_first >= total) return;                                                                    \
  const bool valid = gid0 < total;                                                                    \
  const long gid = valid ? gid0 : total - 1;                                                          \
  const int n = (int)(gid % p.N), b = (int)(gid / p.N);                                               \
  const RowView rv = row_view<HET>(p, b);                                                             \
  const int j0 = rv.jn[n], j1 = rv.jn[n + 1], ns = j1 - j0;                                           \
  const int nsw = warp_max_i(ns);                                                                     \
  const double* ub = p.u + (long)b * rv.us;                                                           \
  const float* ufb = p.uf + (long)b * rv.us;                                                          \
  Cheb<R>& ch = chs[gib];                                                                             \
  int Kw, Sw;                                                                                         \
  cheb_load<G, R>(ch, reinterpret_cast<const Cheb<R>*>(p.cheb) + gid, lg, Kw, Sw);                    \
  Op op;                                                                                              \
  op.load(reinterpret_cast<const R*>(p.H) + rv.hoff, p.H0d + rv.doff, p.d, lg, smem_raw);             \
  op.scale(p.H0d + rv.doff, p.d, lg, ch);                                                             \
  const long off_n = ((long)b * (p.N + 1) + n) * p.d;                                                 \
  R2* zs = reinterpret_cast<R2*>(p.zs) + (long)b * (rv.us + p.N) + j0 + n;                            \
  (void)ub; (void)GE; (void)PK

// ------------------------------------------------------------------------------ k_subfwd
// Algorithm 1 step (c) in the two-trajectory form of the proof of Theorem 2 (first local step, phi =
// phi^u): on sub-interval n, psi_n = a_n psi + b_n chi and chi_n = a_{n+1} psi + b_{n+1} chi with psi,
// chi the global trajectories, so Im<chi_n|H1|psi_n> = Im<chi|H1|psi> / beta_n and J_n's residual is
// (chi - psi)(t_{n+1}) / beta_n.  chi obeys the same propagator as psi, so one group per (problem, n)
// carries BOTH forward from the boundary states psi(t_n), chi(t_n) that steps (a)-(b) stored, and forms
// z_s = <chi_s|H1 psi_s> at every step on the fly: the global trajectories are checkpointed at the
// partition and each segment is recomputed once; nothing per step is stored but z_s.  Neither state
// carries the per-step global phase exp(-i c tau), and the two phases cancel in z_s.  Crank-Nicolson:
// chi's step gives xi_j = A_j^{-1} chi_j (cn_step_fwd_xi), paired with H1 (psi_j + psi_{j+1}).
constexpr int SUB_KR = 10;   // series terms held in registers by the packed sub-interval sweeps

template <typename R, class Op, bool HET = false>
__global__ void __launch_bounds__(128) k_subfwd(KParams p) {
  ISM_SUB_PREAMBLE;
  Vec<R, E> a, alo, c, clo;   // psi and chi (hi + lo in FP32 propagation)
  load_group_state<R, E>(a, alo, p.psin + off_n, p.d, lg);
  load_group_state<R, E>(c, clo, p.chin + off_n, p.d, lg);
  const bool wr = valid && lg == 0;

  if constexpr (PK) {
    VecP<E> pa, pal, pc, pcl;
    to_packed<R, E>(a, alo, pa, pal);
    to_packed<R, E>(c, clo, pc, pcl);
    // over one sub-interval (~10^2 steps) the roundings of the diagonal's and the coefficients' low
    // parts do not accumulate (a ~1e-8 relative change): both are left out (DL = LOC = false)
    float un = ufb[j0];
    auto body = [&](auto step) {
      for (int s = 0; s < nsw; ++s) {
        const bool act = s < ns;
        const float uj = un;
        if (s + 1 < ns) un = __ldg(ufb + j0 + s + 1);
        VecP<E> h;
        op.h1_p(pa, h);
        float zr, zi;
        g_zdot_p<G, E>(pc, h, zr, zi);
        if (act && wr) zs[s] = make_float2(zr, zi);
        VecP<E> wa = pa, wal = pal, wc = pc, wcl = pcl;
        op.set_u(uj, ch, lg);
        step(wa, wal, wc, wcl);
        if (act) { pa = wa; pal = wal; pc = wc; pcl = wcl; }
      }
    };
    if (Kw <= SUB_KR) {   // coefficients in registers
      CoefP<SUB_KR> cp;
      load_coef<SUB_KR, false, true>(cp, ch);
      const int S = ch.S;
      body([&](VecP<E>& x, VecP<E>& xl, VecP<E>& y, VecP<E>& yl) {
        cheb_step_pr2<true, false, false>(x, xl, y, yl, op, cp, Kw, Sw, S);
      });
    } else {
      body([&](VecP<E>& x, VecP<E>& xl, VecP<E>& y, VecP<E>& yl) {
        cheb_step_p2<true, false, false>(x, xl, y, yl, op, ch, Kw, Sw);
      });
    }
    VecP<E> h;
    op.h1_p(pa, h);
    float zr, zi;
    g_zdot_p<G, E>(pc, h, zr, zi);
    if (wr) zs[ns] = make_float2(zr, zi);
  } else if constexpr (Op::CN) {
    Vec<R, E> ha;
    op.h1(a, ha);
    R un = uval<R>(ub, ufb, j0);
    for (int s = 0; s < nsw; ++s) {
      const bool act = s < ns;
      const R uj = un;
      if (s + 1 < ns) un = uval<R>(ub, ufb, j0 + s + 1);
      op.set_u(uj, ch, lg);
      Vec<R, E> wa = a, wc = c, xi, dummy, hb, hs;
      cn_step<false>(wa, dummy, op, ch.h, Kw);
      cn_step_fwd_xi(wc, xi, op, ch.h, Kw);
      op.h1(wa, hb);
#pragma unroll
      for (int r = 0; r < E; ++r) { hs.re[r] = ha.re[r] + hb.re[r]; hs.im[r] = ha.im[r] + hb.im[r]; }
      R zr, zi;
      g_zdot<G, R, E>(xi, hs, zr, zi);
      if (act) {
        a = wa; c = wc; ha = hb;
        if (wr) { R2 z; z.x = zr; z.y = zi; zs[s] = z; }
      }
    }
  } else {
    R un = uval<R>(ub, ufb, j0);
    for (int s = 0; s < nsw; ++s) {
      const bool act = s < ns;
      const R uj = un;
      if (s + 1 < ns) un = uval<R>(ub, ufb, j0 + s + 1);
      Vec<R, E> h;
      op.h1(a, h);
      R zr, zi;
      g_zdot<G, R, E>(c, h, zr, zi);
      if (act && wr) { R2 z; z.x = zr; z.y = zi; zs[s] = z; }
      Vec<R, E> wa = a, wal = alo, wc = c, wcl = clo;
      op.set_u(uj, ch, lg);
      prop_step<false, COMP>(wa, wal, op, ch, Kw, Sw);
      prop_step<false, COMP>(wc, wcl, op, ch, Kw, Sw);
      if (act) { a = wa; alo = wal; c = wc; clo = wcl; }
    }
    Vec<R, E> h;
    op.h1(a, h);
    R zr, zi;
    g_zdot<G, R, E>(c, h, zr, zi);
    if (wr) { R2 z; z.x = zr; z.y = zi; zs[ns] = z; }
  }
  __syncwarp();

  // |delta(t_{n+1})|^2 with delta = (chi - psi)(t_{n+1}) / beta_n from the FP64 boundary states
  const double beta = HET ? p.rt.beta[(long)b * p.N + n] : p.beta[n];
  double nrm = 0.0;
#pragma unroll
  for (int r = 0; r < E; ++r) {
    const int e = lg * E + r;
    if (e < p.d) {
      const double2 x = p.chin[off_n + p.d + e], y = p.psin[off_n + p.d + e];
      const double dr = (x.x - y.x) / beta, di = (x.y - y.y) / beta;
      nrm += dr * dr + di * di;
    }
  }
  nrm = g_sum<G>(nrm);
  sub_grad_pass<G, Op::CN, HET>(p, zs, b, n, gid, j0, ns, 1.0, 0.0, nrm, lg, G, valid);
  if (valid) count_work<R>(p.count, ch, 2L * ns, lg);   // psi and chi forward
}

// ------------------------------------------------------------------------------ k_subinterval
// Algorithm 1 step (c), literal sub-problem (any phi; local steps after the first, and the FP64
// default): per (problem, n) the forward state psi_n from phi_n (Eq. (dirpara)), then the adjoint
// backward from phi_{n+1} (proof of Theorem 2) in the delta form delta = chi_n - psi_n, delta(t_{n+1})
// = phi_{n+1} - psi_n(t_{n+1}) in FP64 (Im<psi|H1|psi> = 0, so Im<chi_n|H1|psi_n> = Im<delta|H1|psi_n>).
// The adjoint needs psi_n at every step in reverse order.  The forward sweep stores psi_n every
// p.cks steps (checkpoints; hi + lo in FP32 propagation, so a recomputation repeats the forward sweep
// bit for bit); the backward sweep runs the segments last to first, recomputing each segment's H1
// psi_n from its checkpoint into a buffer of p.cks slots, then stepping delta back through it.
// Storage per sub-interval: ceil(ns / cks) states and cks H1 psi vectors instead of ns.
template <typename R, class Op>
__global__ void __launch_bounds__(128) k_subinterval(KParams p) {
  constexpr bool HET = false;   // literal sub-problems: plans of one problem kind only
  ISM_SUB_PREAMBLE;
  const int S = p.cks;
  constexpr int CKP = COMP ? 2 : 1;   // checkpoint parts: hi (+ lo)
  R2* ck = reinterpret_cast<R2*>(p.ckpt) + gid * (long)p.nck * CKP * GE + lg * E;   // checkpoint c at ck + c*CKP*GE
  R2* sb = reinterpret_cast<R2*>(p.segb) + gid * (long)S * GE + lg * E;             // segment slot i at sb + i*GE
  // Propagation omits the global phase exp(-i c tau) of each step: over the sub-interval it multiplies
  // psi_n(t_{n+1}) by exp(-i Phi), Phi = c (t_{n+1} - t_n), and every z_s = <delta_s|H1 psi_s> by the
  // same exp(-i Phi) (delta carries exp(+i c (t_{n+1} - t_j)), psi_n exp(-i c (t_j - t_n))); both are
  // applied once, in FP64.
  const double sPhi = ch.sph, cPhi = ch.cph;
  const double2* phn = p.phi + off_n;
  const double2* phn1 = p.phi + off_n + p.d;
  Vec<R, E> v, lo;
  load_group_state<R, E>(v, lo, phn, p.d, lg);
  const bool wr = valid && lg == 0;
  auto put_ck = [&](int c, const Vec<R, E>& x, const Vec<R, E>& xl) {
#pragma unroll
    for (int r = 0; r < E; ++r) {
      R2 z; z.x = x.re[r]; z.y = x.im[r];
      ck[(long)c * CKP * GE + r] = z;
      if (COMP) { R2 y; y.x = xl.re[r]; y.y = xl.im[r]; ck[(long)c * CKP * GE + GE + r] = y; }
    }
  };
  auto get_ck = [&](int c, Vec<R, E>& x, Vec<R, E>& xl) {
#pragma unroll
    for (int r = 0; r < E; ++r) {
      const R2 z = ck[(long)c * CKP * GE + r];
      x.re[r] = z.x; x.im[r] = z.y;
      if (COMP) { const R2 y = ck[(long)c * CKP * GE + GE + r]; xl.re[r] = y.x; xl.im[r] = y.y; }
      else { xl.re[r] = R(0); xl.im[r] = R(0); }
    }
  };
  auto uat = [&](int s) { return uval<R>(p.u + (long)b * rv.us, ufb, j0 + (s < ns ? s : ns - 1)); };

  // ---- forward sweep: checkpoints, then psi_{s+1} = U_s psi_s
  Vec<R, E> hend;   // H1 psi_n(t_{n+1})
  {
    R un = uat(0);
    int cc = 0;
    for (int s = 0; s < nsw; ++s) {
      const bool act = s < ns;
      const R uj = un;
      if (s + 1 < nsw) un = uat(s + 1);
      if (cc == 0 && act && valid) put_ck(s / S, v, lo);
      if (++cc == S) cc = 0;
      Vec<R, E> w = v, wl = lo;
      op.set_u(uj, ch, lg);
      if constexpr (PK) {
        VecP<E> pv, pl;
        to_packed<R, E>(w, wl, pv, pl);
        cheb_step_p<false, true, false, true>(pv, pl, op, ch, Kw, Sw);
#pragma unroll
        for (int r = 0; r < E; ++r) { w.re[r] = pv.z[r].x; w.im[r] = pv.z[r].y; wl.re[r] = pl.z[r].x; wl.im[r] = pl.z[r].y; }
      } else {
        prop_step<false, COMP>(w, wl, op, ch, Kw, Sw);
      }
      if (act) { v = w; lo = wl; }
    }
    op.h1(v, hend);
  }

  // ---- terminal residual delta = phi_{n+1} - psi_n(t_{n+1}) in FP64 (its norm gives J_n)
  double nrm = 0.0;
  Vec<R, E> dl;
#pragma unroll
  for (int r = 0; r < E; ++r) {
    const int e = lg * E + r;
    const double2 z = e < p.d ? phn1[e] : make_double2(0.0, 0.0);
    double pr, pi;
    phase_rotate(cPhi, sPhi, false, (double)v.re[r] + (double)lo.re[r], (double)v.im[r] + (double)lo.im[r], pr, pi);
    double dr = z.x - pr, di = z.y - pi;
    dl.re[r] = (R)dr;
    dl.im[r] = (R)di;
    if (e >= p.d) { dr = 0.0; di = 0.0; }
    nrm += dr * dr + di * di;
  }
  nrm = g_sum<G>(nrm);
  if constexpr (!Op::CN) {
    R zr, zi;
    g_zdot<G, R, E>(dl, hend, zr, zi);
    if (wr) { R2 z; z.x = zr; z.y = zi; zs[ns] = z; }
  }

  // ---- backward sweep over the segments, last to first
  const int nckw = (nsw + S - 1) / S;
  Vec<R, E> hn = hend;   // Crank-Nicolson: H1 psi_{s+1} of the step below
  for (int c = nckw - 1; c >= 0; --c) {
    const int s0 = c * S, s1 = min(s0 + S, nsw);
    // recompute H1 psi_s, s = s0..s1-1, from the checkpoint (bit-identical to the forward sweep)
    {
      Vec<R, E> x, xl;
      get_ck(c, x, xl);
      R un = uat(s0);
      for (int s = s0; s < s1; ++s) {
        const bool act = s < ns;
        const R uj = un;
        if (s + 1 < s1) un = uat(s + 1);
        Vec<R, E> h;
        op.h1(x, h);
        if (act && valid) {
#pragma unroll
          for (int r = 0; r < E; ++r) { R2 z; z.x = h.re[r]; z.y = h.im[r]; sb[(long)(s - s0) * GE + r] = z; }
        }
        if (s + 1 < s1) {
          Vec<R, E> w = x, wl = xl;
          op.set_u(uj, ch, lg);
          if constexpr (PK) {
            VecP<E> pv, pl;
            to_packed<R, E>(w, wl, pv, pl);
            cheb_step_p<false, true, false, true>(pv, pl, op, ch, Kw, Sw);
#pragma unroll
            for (int r = 0; r < E; ++r) { w.re[r] = pv.z[r].x; w.im[r] = pv.z[r].y; wl.re[r] = pl.z[r].x; wl.im[r] = pl.z[r].y; }
          } else {
            prop_step<false, COMP>(w, wl, op, ch, Kw, Sw);
          }
          if (act) { x = w; xl = wl; }
        }
      }
    }
    // delta_s = U_s^H delta_{s+1}; z_s = <delta_s|H1 psi_s> into slot s
    R un = uat(s1 - 1);
    for (int s = s1 - 1; s >= s0; --s) {
      const bool act = s < ns;
      const R uj = un;
      if (s - 1 >= s0) un = uat(s - 1);
      Vec<R, E> hc;
#pragma unroll
      for (int r = 0; r < E; ++r) { const R2 z = sb[(long)(s - s0) * GE + r]; hc.re[r] = z.x; hc.im[r] = z.y; }
      op.set_u(uj, ch, lg);
      Vec<R, E> w = dl;
      R zr, zi;
      if constexpr (Op::CN) {
        // Crank-Nicolson (Sec. 3): lambda_s = A_s xi_s, xi_s = B_s^{-1} lambda_{s+1}; the exact gradient of
        // the discrete J_n pairs xi_s with H1 (psi_s + psi_{s+1}); slot s receives both ends
        Vec<R, E> xi, hs;
        cn_step<true>(w, xi, op, ch.h, Kw);
#pragma unroll
        for (int r = 0; r < E; ++r) { hs.re[r] = hc.re[r] + hn.re[r]; hs.im[r] = hc.im[r] + hn.im[r]; }
        g_zdot<G, R, E>(xi, hs, zr, zi);
      } else if constexpr (PK) {
        VecP<E> pd, dummy, ph;
#pragma unroll
        for (int r = 0; r < E; ++r) { pd.z[r] = make_float2(w.re[r], w.im[r]); ph.z[r] = make_float2(hc.re[r], hc.im[r]); }
        cheb_step_p<true, false, false, false>(pd, dummy, op, ch, Kw, Sw);
#pragma unroll
        for (int r = 0; r < E; ++r) { w.re[r] = pd.z[r].x; w.im[r] = pd.z[r].y; }
        g_zdot_p<G, E>(pd, ph, zr, zi);
      } else {
        cheb_step<true>(w, op, ch, Kw, Sw);
        g_zdot<G, R, E>(w, hc, zr, zi);
      }
      if (act) {
        dl = w;
        hn = hc;
        if (wr) { R2 z; z.x = zr; z.y = zi; zs[s] = z; }
      }
    }
  }
  __syncwarp();
  sub_grad_pass<G, Op::CN, HET>(p, zs, b, n, gid, j0, ns, Op::CN ? 1.0 : cPhi, Op::CN ? 0.0 : sPhi, nrm, lg, G, valid);
  // forward U sweep, its recomputation (every segment but the checkpointed state) and the U^H sweep
  if (valid) count_work<R>(p.count, ch, 3L * ns - (ns + S - 1) / S, lg);
}

__device__ inline double block_sum(double v, double* red) {
  for (int m = 16; m >= 1; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
  return s;
}

// ---------------------------------------------------------------------------- k_cheb_prep
// Per (problem, n): the bound max|u| on the sub-interval, the penalty sum, the FP32 controls and the
// propagator parameters.  Two layouts with the same arithmetic (the same bits): k_cheb_prep_w, one
// warp per pair with lane k evaluating the Bessel series of term k, has the shortest latency for few
// pairs; k_cheb_prep, one warp per pair for the controls and one thread per pair for the parameters,
// does only the terms a sub-interval needs, so for many pairs it is not bound by the FP64 rate.
template <typename R, bool HET = false>
__global__ void __launch_bounds__(32) k_cheb_prep_w(KParams p) {
  const int n = blockIdx.x, b = blockIdx.y, lane = threadIdx.x;
  const RowView rv = row_view<HET>(p, b);
  const int j0 = rv.jn[n], j1 = rv.jn[n + 1];
  const double* ub = p.u + (long)b * rv.us;
  float um = 0.f;   // |u| bound; the margin in cheb_params covers its FP32 rounding
  double pen = 0.0;
  float* ufb = p.uf ? p.uf + (long)b * rv.us : nullptr;
  for (int j = j0 + lane; j < j1; j += 32) {
    const double uj = ub[j];
    if (ufb) ufb[j] = (float)uj;
    um = fmaxf(um, fabsf((float)uj));
    if (rv.alpha) pen += rv.alpha[j] * uj * uj;
  }
  for (int m = 16; m >= 1; m >>= 1) {
    um = fmaxf(um, __shfl_xor_sync(0xffffffffu, um, m));
    pen += __shfl_xor_sync(0xffffffffu, pen, m);
  }
  if (lane == 0 && p.pen) p.pen[(long)b * p.N + n] = pen;
  __shared__ Cheb<R> ch;
  if (p.scheme == 1) {
    if (lane == 0) cn_params<R>(ch, rv.tau, rv.r0, rv.h1n, (double)um, p.tol, p.status);
  } else {
    cheb_params<R>(ch, p.ctab, rv.tau, rv.c0, rv.r0, rv.h1n, (double)um, p.tol, rv.phase[n], p.status);
  }
  __syncwarp();
  const int* s = reinterpret_cast<const int*>(&ch);
  int* d = reinterpret_cast<int*>(const_cast<void*>(p.cheb)) + ((long)b * p.N + n) * (sizeof(Cheb<R>) / sizeof(int));
  for (int i = lane; i < (int)(sizeof(Cheb<R>) / sizeof(int)); i += 32) d[i] = s[i];
}

// (problem, sub-interval) pairs per block of k_cheb_prep; up to CHEB_WARP_PAIRS pairs per launch the
// warp-per-pair layout runs instead
constexpr int CHEB_PAIRS = 32;
constexpr long CHEB_WARP_PAIRS = 8192;

template <typename R, bool HET = false>
__global__ void __launch_bounds__(128) k_cheb_prep(KParams p) {
  __shared__ Cheb<R> chs[CHEB_PAIRS];
  __shared__ double sa[CHEB_PAIRS][KMAX];
  __shared__ float sum_[CHEB_PAIRS];
  const long total = (long)p.B * p.N, i0 = (long)blockIdx.x * CHEB_PAIRS;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // (1) one warp per pair: the |u| bound, the penalty sum and the FP32 controls (coalesced reads)
  for (int q = w; q < CHEB_PAIRS; q += 4) {
    const long i = i0 + q;
    if (i >= total) break;   // warp-uniform
    const int b = (int)(i / p.N), n = (int)(i % p.N);
    const RowView rv = row_view<HET>(p, b);
    const int j0 = rv.jn[n], j1 = rv.jn[n + 1];
    const double* ub = p.u + (long)b * rv.us;
    float um = 0.f;   // |u| bound; the margin in the parameters covers its FP32 rounding
    double pen = 0.0;
    float* ufb = p.uf ? p.uf + (long)b * rv.us : nullptr;
    for (int j = j0 + lane; j < j1; j += 32) {
      const double uj = ub[j];
      if (ufb) ufb[j] = (float)uj;
      um = fmaxf(um, fabsf((float)uj));
      if (rv.alpha) pen += rv.alpha[j] * uj * uj;
    }
    for (int m = 16; m >= 1; m >>= 1) {
      um = fmaxf(um, __shfl_xor_sync(0xffffffffu, um, m));
      pen += __shfl_xor_sync(0xffffffffu, pen, m);
    }
    if (lane == 0) {
      if (p.pen) p.pen[i] = pen;
      sum_[q] = um;
    }
  }
  __syncthreads();
  // (2) one thread per pair: the propagator parameters (FP64 work per pair, not per lane)
  if (w == 0 && i0 + lane < total) {
    const long i = i0 + lane;
    const int b = (int)(i / p.N), n = (int)(i % p.N);
    const RowView rv = row_view<HET>(p, b);
    if (p.scheme == 1) cn_params<R>(chs[lane], rv.tau, rv.r0, rv.h1n, (double)sum_[lane], p.tol, p.status);
    else cheb_params_1<R>(chs[lane], sa[lane], p.ctab, rv.tau, rv.c0, rv.r0, rv.h1n, (double)sum_[lane], p.tol,
                          rv.phase[n], p.status);
  }
  __syncthreads();
  // (3) the pairs' parameters out, as consecutive words
  constexpr int words = sizeof(Cheb<R>) / sizeof(int);
  const long np = total - i0 < CHEB_PAIRS ? total - i0 : CHEB_PAIRS;
  const int* src = reinterpret_cast<const int*>(chs);
  int* dst = reinterpret_cast<int*>(const_cast<void*>(p.cheb)) + i0 * words;
  for (long x = threadIdx.x; x < np * words; x += blockDim.x) dst[x] = src[x];
}

// ---------------------------------------------------------------------- k_sweeps2 / k_gradpass
// Theorem 2 (two-trajectory) form of the first local step, with the two sweeps run concurrently:
// blockIdx.y = 0 propagates psi forward from psi(t_n) (compensated) and stores H1 psi^_j in trajectory
// slot j - j_n (0..ns); blockIdx.y = 1 propagates chi backward from chi(t_{n+1}) and stores chi^_j in a
// second trajectory (slot 0..ns).  Neither depends on the other.  k_gradpass then forms every
// <chi^_j|H1 psi^_j>, the gradient, Err, J_n and the ascent step in parallel over steps.
template <typename R, class Op>
__global__ void __launch_bounds__(128) k_sweeps2(KParams p) {
  constexpr int G = Op::G, E = Op::E, GPB = 128 / G, GE = G * E;
  constexpr bool COMP = sizeof(R) == 4;
  using R2 = typename C2<R>::T;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ Cheb<R> chs[GPB];
  const int lg = threadIdx.x % G, gib = threadIdx.x / G;
  const long gid0 = (long)blockIdx.x * GPB + gib;
  const long total = (long)p.B * p.N;
  const bool fwd = blockIdx.y == 0;
  if (Op::G * Op::E == Op::DP_SMEM) {
    const R* src = reinterpret_cast<const R*>(p.H);
    R* dst = reinterpret_cast<R*>(smem_raw);
    for (int i = threadIdx.x; i < Op::SMEM_WORDS; i += blockDim.x) dst[i] = src[i];
    __syncthreads();
  }
  const long warp_first = ((long)blockIdx.x * GPB + (threadIdx.x / 32) * (32 / G));
  if (warp_first >= total) return;
  const bool valid = gid0 < total;
  const long gid = valid ? gid0 : total - 1;
  const int n = (int)(gid % p.N), b = (int)(gid / p.N);
  const int j0 = p.jn[n], j1 = p.jn[n + 1], ns = j1 - j0;
  const int nsw = warp_max_i(ns);
  const double* ub = p.u + (long)b * p.Nt;
  const float* ufb = p.uf + (long)b * p.Nt;

  Cheb<R>& ch = chs[gib];
  int Kw, Sw;
  cheb_load<G, R>(ch, reinterpret_cast<const Cheb<R>*>(p.cheb) + gid, lg, Kw, Sw);
  Op op;
  op.load(reinterpret_cast<const R*>(p.H), p.H0d, p.d, lg, smem_raw);
  op.scale(p.H0d, p.d, lg, ch);

  const long off_n = ((long)b * (p.N + 1) + n) * p.d;
  const double2* st = fwd ? p.psin + off_n : p.chin + off_n + p.d;
  Vec<R, E> v, lo;
#pragma unroll
  for (int r = 0; r < E; ++r) {
    int e = lg * E + r;
    double2 z = e < p.d ? st[e] : make_double2(0.0, 0.0);
    v.re[r] = (R)z.x;
    v.im[r] = (R)z.y;
    lo.re[r] = COMP ? (R)(z.x - (double)v.re[r]) : R(0);
    lo.im[r] = COMP ? (R)(z.y - (double)v.im[r]) : R(0);
  }
  R2* tr = reinterpret_cast<R2*>(fwd ? p.traj : p.traj2) + ((long)b * (p.Nt + p.N) + j0 + n) * GE + lg * E;
  if constexpr (sizeof(R) == 4 && Op::PACKED) {   // packed FP32: both halves per instruction
    VecP<E> pv, pl;
#pragma unroll
    for (int r = 0; r < E; ++r) {
      pv.z[r] = make_float2(v.re[r], v.im[r]);
      pl.z[r] = make_float2(lo.re[r], lo.im[r]);
    }
    float2* trp = reinterpret_cast<float2*>(tr);
    auto putp = [&](int slot, const VecP<E>& x) {
      if (valid) {
#pragma unroll
        for (int r = 0; r < E; ++r) trp[(long)slot * GE + r] = x.z[r];
      }
    };
    if (fwd) {
      float ua = ufb[j0], ub1 = ns > 1 ? ufb[j0 + 1] : ua;
      for (int s = 0; s < nsw; ++s) {
        const bool act = s < ns;
        const float uj = ua;
        ua = ub1;
        if (s + 2 < ns) ub1 = ufb[j0 + s + 2];
        VecP<E> hv;
        op.h1_p(pv, hv);
        if (act) putp(s, hv);
        VecP<E> w = pv, wl = pl;
        op.set_u(uj, ch, lg);
        cheb_step_p<false, true, false, true>(w, wl, op, ch, Kw, Sw);
        if (act) { pv = w; pl = wl; }
      }
      VecP<E> hv;
      op.h1_p(pv, hv);
      putp(ns, hv);
    } else {
      putp(ns, pv);
      const int top = ns - 1;
      float ua = ufb[j0 + top], ub1 = ufb[j0 + (top > 0 ? top - 1 : top)];
      for (int s = nsw - 1; s >= 0; --s) {
        const bool act = s < ns;
        const float uj = ua;
        if (act) {
          ua = ub1;
          if (s - 2 >= 0) ub1 = ufb[j0 + s - 2];
        }
        VecP<E> w = pv, wl = pl;
        op.set_u(uj, ch, lg);
        cheb_step_p<true, true, false, false>(w, wl, op, ch, Kw, Sw);
        if (act) { pv = w; pl = wl; putp(s, pv); }
      }
    }
  } else {
    auto put = [&](int slot, const Vec<R, E>& x) {
      if (valid) {
  #pragma unroll
        for (int r = 0; r < E; ++r) { R2 z; z.x = x.re[r]; z.y = x.im[r]; tr[(long)slot * GE + r] = z; }
      }
    };
    if (fwd) {
      R ua = uval<R>(ub, ufb, j0), ub1 = ns > 1 ? uval<R>(ub, ufb, j0 + 1) : ua;
      for (int s = 0; s < nsw; ++s) {
        const bool act = s < ns;
        const R uj = ua;
        ua = ub1;
        if (s + 2 < ns) ub1 = uval<R>(ub, ufb, j0 + s + 2);
        Vec<R, E> hv;
        op.h1(v, hv);
        if (act) put(s, hv);
        Vec<R, E> w = v, wl = lo;
        op.set_u(uj, ch, lg);
        cheb_step<false, COMP>(w, wl, op, ch, Kw, Sw);
        if (act) { v = w; lo = wl; }
      }
      Vec<R, E> hv;
      op.h1(v, hv);
      put(ns, hv);
    } else {
      put(ns, v);
      const int top = ns - 1;
      R ua = uval<R>(ub, ufb, j0 + top), ub1 = uval<R>(ub, ufb, j0 + (top > 0 ? top - 1 : top));
      for (int s = nsw - 1; s >= 0; --s) {
        const bool act = s < ns;
        const R uj = ua;
        if (act) {
          ua = ub1;
          if (s - 2 >= 0) ub1 = uval<R>(ub, ufb, j0 + s - 2);
        }
        Vec<R, E> w = v, wl = lo;
        op.set_u(uj, ch, lg);
        cheb_step<true, COMP>(w, wl, op, ch, Kw, Sw);
        if (act) { v = w; lo = wl; put(s, v); }
      }
    }
  }
  if (valid) count_work<R>(p.count, ch, ns, lg);
}

// ------------------------------------------------------------------------------ k_gsweep
// Algorithm 1 steps (a)-(b) by direct propagation, one group per trajectory: psi forward over all Nt
// steps from psi_i and chi backward from chi(T), psi(t_n) and chi(t_n) stored in FP64 with each
// sub-interval's phase applied in FP64 there (the states continue from their FP64 values).  Work
// 2 Nt state-steps per problem instead of the assembly's d Nt, but Nt sequential steps: the choice
// for many problems per launch, where the groups of different problems fill the GPU.
// grid (ceil(B / groups per CTA), nch): blockIdx.y is the direction, so every warp runs one
// direction (the group shuffles and warp barriers need the whole warp on the same path).  Direction 1
// (chi) exists only for the overlap objective; the observable objective runs chi after psi in the
// same group (chi(T) = O psi(T) needs psi(T)).
constexpr int GSWEEP_KR = 10;   // series terms held in registers by the packed direct sweeps

template <typename R, class Op, bool HET = false>
__global__ void __launch_bounds__(128) k_gsweep(KParams p) {
  constexpr int G = Op::G, E = Op::E, GPB = 128 / G;
  constexpr bool COMP = sizeof(R) == 4;
  constexpr bool PK = sizeof(R) == 4 && Op::PACKED;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ Cheb<R> chs[GPB];
  const int lg = threadIdx.x % G, gib = threadIdx.x / G;
  const int nch = gridDim.y;
  const long gid0 = (long)blockIdx.x * GPB + gib;
  const long total = (long)p.B;
  if (Op::G * Op::E == Op::DP_SMEM) {
    const R* src = reinterpret_cast<const R*>(p.H);
    R* dst = reinterpret_cast<R*>(smem_raw);
    for (int i = threadIdx.x; i < Op::SMEM_WORDS; i += blockDim.x) dst[i] = src[i];
    __syncthreads();
  }
  const long warp_first = ((long)blockIdx.x * GPB + (threadIdx.x / 32) * (32 / G));
  if (warp_first >= total) return;
  const bool valid = gid0 < total;
  const long gid = valid ? gid0 : total - 1;
  const int b = (int)gid, dir = (int)blockIdx.y;
  const int d = p.d, N = p.N;
  const RowView rv = row_view<HET>(p, b);
  const double* ub = p.u + (long)b * rv.us;
  const float* ufb = p.uf + (long)b * rv.us;
  const double2* psi_i = p.psi_i + rv.doff;
  const double2* psi_f = p.psi_f + rv.doff;
  double2* psin = p.psin_w + (long)b * (N + 1) * d;
  double2* chin = p.chin_w + (long)b * (N + 1) * d;
  Cheb<R>& ch = chs[gib];
  Op op;
  op.load(reinterpret_cast<const R*>(p.H) + rv.hoff, p.H0d + rv.doff, d, lg, smem_raw);
  Vec<R, E> v, lo;
  auto load64 = [&](const double2* src) {
#pragma unroll
    for (int r = 0; r < E; ++r) {
      const int e = lg * E + r;
      const double2 z = e < d ? src[e] : make_double2(0.0, 0.0);
      v.re[r] = (R)z.x;
      v.im[r] = (R)z.y;
      lo.re[r] = COMP ? (R)(z.x - (double)v.re[r]) : R(0);
      lo.im[r] = COMP ? (R)(z.y - (double)v.im[r]) : R(0);
    }
  };
  // segment phase in FP64, store, continue from it; the FP64 squared norm goes to nslot (for the
  // renormalisation in k_phi, which then reads one number instead of summing the state again)
  auto store64 = [&](bool adj, double2* dst, double* nslot) {
    double sq = 0.0;
#pragma unroll
    for (int r = 0; r < E; ++r) {
      const int e = lg * E + r;
      double yr, yi;
      phase_rotate(ch.cph, ch.sph, adj, (double)v.re[r] + (double)lo.re[r], (double)v.im[r] + (double)lo.im[r], yr, yi);
      if (e < d) {
        if (valid) dst[e] = make_double2(yr, yi);
        sq = fma(yr, yr, fma(yi, yi, sq));
      }
      v.re[r] = (R)yr;
      v.im[r] = (R)yi;
      lo.re[r] = COMP ? (R)(yr - (double)v.re[r]) : R(0);
      lo.im[r] = COMP ? (R)(yi - (double)v.im[r]) : R(0);
    }
    sq = g_sum<G>(sq);
    if (nslot && valid && lg == 0) *nslot = sq;
  };
  double* nrm = p.nrm_w ? p.nrm_w + (long)b * (N + 1) * 2 : nullptr;   // [N+1][2]: |psi(t_n)|^2, |chi(t_n)|^2
  // propagate over sub-interval n forward (ADJ = false) or backward (ADJ = true)
  auto segment = [&](int n, auto adj_tag) {
    constexpr bool ADJ = decltype(adj_tag)::value;
    int Kw, Sw;
    __syncwarp();
    cheb_load<G, R>(ch, reinterpret_cast<const Cheb<R>*>(p.cheb) + (long)b * N + n, lg, Kw, Sw);
    op.scale(p.H0d + rv.doff, d, lg, ch);
    const int j0 = rv.jn[n], j1 = rv.jn[n + 1];
    // Heterogeneous batches: the groups of a warp belong to different problems whose sub-intervals
    // have different step counts; the warp runs the largest count (the group shuffles need every lane)
    // and a group's steps beyond its own are computed and discarded.
    const int ns = j1 - j0;
    const int nsw = HET ? warp_max_i(ns) : ns;
    if constexpr (PK) {
      VecP<E> pv, pl;
#pragma unroll
      for (int r = 0; r < E; ++r) { pv.z[r] = make_float2(v.re[r], v.im[r]); pl.z[r] = make_float2(lo.re[r], lo.im[r]); }
      // controls two steps ahead in registers: the sweep's steps are its critical path
      auto jof = [&](int s) { return ADJ ? j1 - 1 - s : j0 + s; };
      float ua = __ldg(ufb + jof(0)), ub1 = ns > 1 ? __ldg(ufb + jof(1)) : 0.f;
      if (Kw <= GSWEEP_KR) {   // coefficients in registers
        CoefP<GSWEEP_KR> cp;
        load_coef<GSWEEP_KR, ADJ, true>(cp, ch);
        const int S = ch.S;
        for (int s = 0; s < nsw; ++s) {
          const float uj = ua;
          ua = ub1;
          if (s + 2 < ns) ub1 = __ldg(ufb + jof(s + 2));
          op.set_u(uj, ch, lg);
          if constexpr (HET) {
            VecP<E> w = pv, wl = pl;
            cheb_step_pr<true>(w, wl, op, cp, Kw, Sw, S);
            if (s < ns) { pv = w; pl = wl; }
          } else {
            cheb_step_pr<true>(pv, pl, op, cp, Kw, Sw, S);
          }
        }
      } else {
        for (int s = 0; s < nsw; ++s) {
          const float uj = ua;
          ua = ub1;
          if (s + 2 < ns) ub1 = __ldg(ufb + jof(s + 2));
          op.set_u(uj, ch, lg);
          if constexpr (HET) {
            VecP<E> w = pv, wl = pl;
            cheb_step_p<ADJ, true>(w, wl, op, ch, Kw, Sw);
            if (s < ns) { pv = w; pl = wl; }
          } else {
            cheb_step_p<ADJ, true>(pv, pl, op, ch, Kw, Sw);
          }
        }
      }
#pragma unroll
      for (int r = 0; r < E; ++r) { v.re[r] = pv.z[r].x; v.im[r] = pv.z[r].y; lo.re[r] = pl.z[r].x; lo.im[r] = pl.z[r].y; }
    } else {
      auto jof = [&](int s) { return ADJ ? j1 - 1 - s : j0 + s; };
      R ua = uval<R>(ub, ufb, jof(0)), ub1 = ns > 1 ? uval<R>(ub, ufb, jof(1)) : R(0);
      for (int s = 0; s < nsw; ++s) {
        const R uj = ua;
        ua = ub1;
        if (s + 2 < ns) ub1 = uval<R>(ub, ufb, jof(s + 2));
        op.set_u(uj, ch, lg);
        if constexpr (HET) {
          Vec<R, E> w = v, wl = lo;
          prop_step<ADJ, COMP>(w, wl, op, ch, Kw, Sw);
          if (s < ns) { v = w; lo = wl; }
        } else {
          prop_step<ADJ, COMP>(v, lo, op, ch, Kw, Sw);
        }
      }
    }
    if (valid) count_work<R>(p.count, ch, j1 - j0, lg);
  };
  if (dir == 0) {
    load64(psi_i);
    if (valid)
      for (int e = lg; e < d; e += G) psin[e] = psi_i[e];
    for (int n = 0; n < N; ++n) {
      segment(n, std::false_type());
      store64(false, psin + (long)(n + 1) * d, nrm ? nrm + 2 * (n + 1) : nullptr);
    }
  }
  if (dir == 1 || nch == 1) {
    double2* chT = chin + (long)N * d;
    if (p.obj == 0) {
      if (valid)
        for (int e = lg; e < d; e += G) chT[e] = psi_f[e];
    } else {   // chi(T) = O psi(T) in FP64; psi(T) was stored by this group
      __syncwarp();
      const double2* psT = psin + (long)N * d;
      for (int e = lg; e < d; e += G) {
        double sr = 0.0, si = 0.0;
        for (int f = 0; f < d; ++f) {
          const double o = p.O[(HET ? (long)b * d * d : 0L) + (long)e * d + f];
          const double2 z = psT[f];
          sr = fma(o, z.x, sr);
          si = fma(o, z.y, si);
        }
        if (valid) chT[e] = make_double2(sr, si);
      }
      __syncwarp();
      double sq = 0.0;
      for (int e = lg; e < d; e += G) {
        const double2 z = chT[e];
        sq = fma(z.x, z.x, fma(z.y, z.y, sq));
      }
      sq = g_sum<G>(sq);
      if (nrm && valid && lg == 0) nrm[2 * N + 1] = sq;
    }
    __syncwarp();
    load64(chT);
    for (int n = N - 1; n >= 0; --n) {
      segment(n, std::true_type());
      store64(true, chin + (long)n * d, nrm ? nrm + 2 * n + 1 : nullptr);
    }
  }
}

// One block per (problem, n); threads over the steps of the sub-interval.
template <typename R>
__global__ void __launch_bounds__(256) k_gradpass(KParams p, int GE) {
  using R2 = typename C2<R>::T;
  __shared__ double red[8];
  const int b = blockIdx.y, n = blockIdx.x, t = threadIdx.x, d = p.d;
  const int j0 = p.jn[n], j1 = p.jn[n + 1], ns = j1 - j0;
  const double beta = p.beta[n];
  const long base = ((long)b * (p.Nt + p.N) + j0 + n) * GE;
  const R2* hp = reinterpret_cast<const R2*>(p.traj) + base;    // H1 psi^ per slot
  const R2* cp = reinterpret_cast<const R2*>(p.traj2) + base;   // chi^ per slot
  const Cheb<R>& chp = reinterpret_cast<const Cheb<R>*>(p.cheb)[(long)b * p.N + n];
  const double sPhi = chp.sph, cPhi = chp.cph;
  auto I_at = [&](int slot) {   // Im(exp(-i Phi) <chi^|H1 psi^>) at a slot, FP32 products
    R zr = R(0), zi = R(0);
    const R2* h = hp + (long)slot * GE;
    const R2* c = cp + (long)slot * GE;
    for (int e = 0; e < d; ++e) {
      const R2 a = c[e], y = h[e];
      zr = fma(a.x, y.x, fma(a.y, y.y, zr));
      zi = fma(a.x, y.y, fma(-a.y, y.x, zi));
    }
    return cPhi * (double)zi - sPhi * (double)zr;
  };
  const double bs = p.global ? 1.0 : beta;   // Theorem 2: beta_n g_n is the gradient of J
  const double ht = 0.5 * p.tau * p.w / bs, tb = p.tau / bs, step = p.rho * beta / p.tau;
  double* ub = p.u + (long)b * p.Nt;
  double* gb = p.grad + (long)b * p.Nt;
  double err = 0.0, pen = 0.0;
  for (int s = t; s < ns; s += blockDim.x) {
    const int j = j0 + s;
    const double uj = ub[j];
    const double al = p.alpha ? p.alpha[j] : 0.0;
    const double g = ht * (I_at(s) + I_at(s + 1)) - tb * al * uj;
    err += fabs(g);
    pen += al * uj * uj;
    gb[j] = g;
    if (p.update) ub[j] = uj + step * g;
  }
  double nrm = 0.0;   // J_n: delta = (chi - psi)(t_{n+1}) / beta_n from the chain (FP64)
  const long off = ((long)b * (p.N + 1) + n + 1) * d;
  for (int e = t; e < d; e += blockDim.x) {
    const double2 c = p.chin[off + e], ps = p.psin[off + e];
    const double dr = (c.x - ps.x) / beta, di = (c.y - ps.y) / beta;
    nrm += dr * dr + di * di;
  }
  err = block_sum(err, red);
  pen = block_sum(pen, red);
  nrm = block_sum(nrm, red);
  if (t == 0) {
    const long id = (long)b * p.N + n;
    if (p.Jn) p.Jn[id] = p.w * (-0.5 * nrm) - 0.5 * tb * pen;
    if (p.err) p.err[id] = err;
  }
}

// -------------------------------------------------------------------------------- k_chain
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// One elected thread: expect `bytes` on `bar` and start the bulk copy global -> shared.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// Bounded wait on phase `parity`; returns false when the cap is reached.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, int max_spin) {
  for (int it = 0; it < max_spin; ++it) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
    if (it > 64) __nanosleep(64);
  }
  return false;
}


// ---------------------------------------------------------------------------------- chains
// The chain is a sequence of 2N small dependent matvecs: latency, not bandwidth.  The block is warp
// specialised.  One producer warp streams the tiles M_n (left in L2 by the assembly) into a ring of NS
// shared-memory stages with TMA bulk copies: before refilling a stage it waits on that stage's "empty"
// mbarrier, on which each consumer warp arrives once it has read the tile.  The CW consumer warps wait
// on the stage's "full" mbarrier themselves (every thread, bounded), so no thread carries the copy
// bookkeeping inside the dependent chain, and one named barrier over the consumers per matvec publishes
// the new state.  Consumer thread t owns output row i = t / 8 and the columns k = t (mod 8); three
// shuffles finish each row.
constexpr int CHAIN_MAX_STAGES = 16;
constexpr int CHAIN_DRAIN_SPIN = 1 << 22;   // bounded wait for copies in flight (~0.3 s at most)
constexpr int CHAIN_LANES = 8;      // lanes per output row
constexpr int CHAIN_MAX_THREADS = (64 * CHAIN_LANES / 32 + 1) * 32;

__host__ __device__ inline int chain_consumer_warps(int d) { return (d * CHAIN_LANES + 31) / 32; }

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void consumer_sync(int nthreads) {
  asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory");
}

// Per-thread shared-memory offsets of the tile elements a consumer thread reads, computed once:
// thread (i = t / 8, q = t % 8) reads columns k = q + 8 j, j < JC = ceil(d / 8), of row i.
template <int JC>
struct ChainIdx {
  int off[JC];    // element offset in a tile: (k, i) of M (HERM = false) or (i, k) (HERM = true)
  int xk[JC];     // k
  unsigned on;    // bit j: k < d and i < d
  __device__ void init(int d, int ldm, bool herm) {
    const int i = threadIdx.x / CHAIN_LANES, q = threadIdx.x % CHAIN_LANES;
    on = 0u;
#pragma unroll
    for (int j = 0; j < JC; ++j) {
      const int k = q + CHAIN_LANES * j;
      const bool ok = k < d && i < d;
      off[j] = ok ? (herm ? i * ldm + k : k * ldm + i) : 0;
      xk[j] = ok ? k : 0;
      on |= ok ? (1u << j) : 0u;
    }
  }
};

template <typename R, bool HERM, int JC>
__device__ __forceinline__ void chain_mv(const typename C2<R>::T* Ms, const typename C2<R>::T* x,
                                         typename C2<R>::T* y, const ChainIdx<JC>& ix, int d) {
  using R2 = typename C2<R>::T;
  const int i = threadIdx.x / CHAIN_LANES, q = threadIdx.x % CHAIN_LANES;
  R ar0 = R(0), ai0 = R(0), ar1 = R(0), ai1 = R(0);
#pragma unroll
  for (int j = 0; j < JC; ++j) {
    if (ix.on & (1u << j)) {
      const R2 m = Ms[ix.off[j]];
      const R2 xv = x[ix.xk[j]];
      R& ar = (j & 1) ? ar1 : ar0;
      R& ai = (j & 1) ? ai1 : ai0;
      if (!HERM) { ar = fma(m.x, xv.x, fma(-m.y, xv.y, ar)); ai = fma(m.x, xv.y, fma(m.y, xv.x, ai)); }
      else { ar = fma(m.x, xv.x, fma(m.y, xv.y, ar)); ai = fma(m.x, xv.y, fma(-m.y, xv.x, ai)); }
    }
  }
  R ar = ar0 + ar1, ai = ai0 + ai1;
#pragma unroll
  for (int m = 1; m < CHAIN_LANES; m <<= 1) {
    ar += __shfl_xor_sync(0xffffffffu, ar, m);
    ai += __shfl_xor_sync(0xffffffffu, ai, m);
  }
  if (q == 0 && i < d) { R2 z; z.x = ar; z.y = ai; y[i] = z; }
}

// The ring: use m (0..U-1) of the chain(s) this CTA runs reads tile tile_of(m) from stage m % NS.
template <typename R>
struct ChainRing {
  using R2 = typename C2<R>::T;
  R2* stages;
  uint64_t* full;    // [NS] completes when the copy of a use has landed (count 1 + tx bytes)
  uint64_t* empty;   // [NS] completes when all consumer warps have read a use (count CW)
  const R2* Mb;
  long tst;
  unsigned bytes;
  int NS, U, N, first;   // tile_of(m): first == 0 -> m < N ? m : 2N-1-m; first == 1 -> N-1-m
  __device__ int tile_of(int m) const { return first == 1 ? N - 1 - m : (m < N ? m : 2 * N - 1 - m); }
  __device__ const R2* tile(int m) const { return stages + (m % NS) * tst; }
};

// Producer (lane 0 of the last warp): issue every use in order, each after its stage has been emptied.
// If an empty-wait gives up (the consumers stopped), stop issuing and wait, bounded, for the copies
// already in flight so that none lands after the block exits.
template <typename R>
__device__ void chain_produce(const ChainRing<R>& ring, int* status, int max_spin) {
  int issued = 0;
  for (int m = 0; m < ring.U; ++m) {
    const int st = m % ring.NS;
    if (m >= ring.NS && !mbar_wait(&ring.empty[st], (unsigned)((m / ring.NS - 1) & 1), max_spin)) {
      atomicOr(status, ST_TIMEOUT);
      break;
    }
    fence_proxy_async();   // the consumers' reads of this stage precede the copy that overwrites it
    bulk_load(ring.stages + st * ring.tst, ring.Mb + (long)ring.tile_of(m) * ring.tst, ring.bytes, &ring.full[st]);
    issued = m + 1;
  }
  // the drain has its own bound, independent of the caller's wait cap: copies in flight complete
  // within microseconds, and none may land after the block exits.  A drain that gives up leaves
  // ST_TIMEOUT (the call then reports ISM_ETIMEOUT and the caller should not reuse the context).
  if (issued < ring.U)
    for (int m = issued - ring.NS < 0 ? 0 : issued - ring.NS; m < issued; ++m)
      if (!mbar_wait(&ring.full[m % ring.NS], (unsigned)((m / ring.NS) & 1), CHAIN_DRAIN_SPIN))
        atomicOr(status, ST_TIMEOUT);
}

// One chain of N matvecs over uses m0 .. m0+N-1 of the ring, run by the CW consumer warps; x_0 in
// xs[0]; stores the N results (FP32 staging) into out[idx * d] with idx = c (psi) or N - c (chi).
// Returns false (uniformly over the consumers) if a tile did not arrive.
// A coarse chain (blocked, sblk > 1) stores its result c at index min(c sblk, Nfull).
template <typename R, bool HERM, int JC>
__device__ bool run_chain(const ChainRing<R>& ring, int m0, int N, int d, int ldm, typename C2<R>::T (*xs)[64],
                          typename C2<R>::T* out, int* fail, int* status, int max_spin, int ncons, int sblk,
                          int Nfull) {
  const int t = threadIdx.x;
  ChainIdx<JC> ix;
  ix.init(d, ldm, HERM);
  for (int c = 0; c <= N; ++c) {
    const int m = m0 + c;
    if (c < N && !mbar_wait(&ring.full[m % ring.NS], (unsigned)((m / ring.NS) & 1), max_spin)) {
      atomicOr(status, ST_TIMEOUT);
      *(volatile int*)fail = 1;
    }
    consumer_sync(ncons);   // result of matvec c-1 visible; every consumer has waited for tile m
    if (*(volatile int*)fail) return false;
    if (c >= 1) {
      const int ic = (HERM ? N - c : c) * sblk;
      const int idx = ic < Nfull ? ic : Nfull;
      if (t < d) out[(long)idx * d + t] = xs[c & 1][t];   // FP32 here; FP64 conversion in k_phi
    }
    if (c < N) {
      chain_mv<R, HERM, JC>(ring.tile(m), xs[c & 1], xs[(c + 1) & 1], ix, d);
      __syncwarp();
      if ((t & 31) == 0) mbar_arrive(&ring.empty[m % ring.NS]);
    }
  }
  consumer_sync(ncons);   // the last stored state is read by other threads next
  return true;
}

// grid (nchains, B), (CW + 1) warps, dynamic shared memory NS tiles.  nchains = 2 (overlap objective):
// CTA 0 runs the psi chain, CTA 1 the chi chain from psi_f, concurrently.  nchains = 1 (observable):
// one CTA runs the psi chain, forms chi(T) = O psi(T) in FP64 and runs the chi chain, all from one ring.
// Intermediate states and J follow in k_phi.
template <typename R, int JC>
__global__ void __launch_bounds__(CHAIN_MAX_THREADS) k_chain(ChainParams p) {
  using R2 = typename C2<R>::T;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full[CHAIN_MAX_STAGES];
  __shared__ __align__(8) uint64_t empty[CHAIN_MAX_STAGES];
  __shared__ __align__(16) R2 xs[2][64];
  __shared__ double2 vd[64];
  __shared__ int fail;
  const int b = blockIdx.y, t = threadIdx.x, d = p.d, N = p.N;
  const int Nn = p.Nc ? p.Nc : N, sb = p.Nc ? p.sblk : 1;   // coarse chain over block products, or plain
  const int cw = chain_consumer_warps(d), ncons = cw * 32;
  double2* chin = p.chin + (long)b * (N + 1) * d;
  const bool single = gridDim.x == 1;
  const bool do_psi = single || blockIdx.x == 0;
  const bool do_chi = single || blockIdx.x == 1;
  ChainRing<R> ring;
  ring.stages = reinterpret_cast<R2*>(smem_raw);
  ring.full = full;
  ring.empty = empty;
  ring.Mb = reinterpret_cast<const R2*>(p.Nc ? p.Mc : p.M) + (long)b * Nn * p.tile_stride;
  ring.tst = p.tile_stride;
  ring.bytes = (unsigned)(p.tile_stride * sizeof(R2));
  ring.NS = p.stages;
  ring.N = Nn;
  ring.U = single ? 2 * Nn : Nn;
  ring.first = (!single && blockIdx.x == 1) ? 1 : 0;
  if (t == 0) {
    fail = 0;
    for (int i = 0; i < ring.NS; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], (unsigned)cw);
    }
    fence_mbar_init();
  }
  __syncthreads();   // the last block-wide barrier: producer and consumers part here
  if (t >= ncons) {
    if (t == ncons) chain_produce<R>(ring, p.status, p.max_spin);
    return;
  }

  R2* sps = reinterpret_cast<R2*>(p.stage) + (long)b * 2 * (N + 1) * d;
  R2* sch = sps + (long)(N + 1) * d;
  int m0 = 0;
  if (do_psi) {
    if (t < d) { const double2 z = p.psi_i[t]; R2 r; r.x = (R)z.x; r.y = (R)z.y; xs[0][t] = r; }
    if (!run_chain<R, false, JC>(ring, m0, Nn, d, p.ldm, xs, sps, &fail, p.status, p.max_spin, ncons, sb, N)) return;
    m0 += Nn;
  }
  if (do_chi) {
    if (p.obj == 0) {
      if (t < d) vd[t] = p.psi_f[t];
    } else {   // chi(T) = O psi(T) in FP64 from the FP32 psi(T) in xs[N & 1]
      const int i = t / CHAIN_LANES, q = t % CHAIN_LANES;
      double sr = 0.0, si = 0.0;
      if (i < d)
        for (int k = q; k < d; k += CHAIN_LANES) {
          const double o = p.O[i * d + k];
          const R2 v = xs[Nn & 1][k];
          sr += o * (double)v.x;
          si += o * (double)v.y;
        }
#pragma unroll
      for (int m = 1; m < CHAIN_LANES; m <<= 1) {
        sr += __shfl_xor_sync(0xffffffffu, sr, m);
        si += __shfl_xor_sync(0xffffffffu, si, m);
      }
      if (q == 0 && i < d) vd[i] = make_double2(sr, si);
    }
    consumer_sync(ncons);
    if (t < d) { const double2 z = vd[t]; R2 r; r.x = (R)z.x; r.y = (R)z.y; xs[0][t] = r; chin[(long)N * d + t] = z; }
    if (!run_chain<R, true, JC>(ring, m0, Nn, d, p.ldm, xs, sch, &fail, p.status, p.max_spin, ncons, sb, N)) return;
  }
}


// ------------------------------------------------------------------------ blocked chain
// The chain's 2N dependent matvecs take ~0.4-0.5 us each on one SM.  With N large the chain is
// shortened by products of consecutive propagators (Sec. 3: M_n are products of step propagators
// too): k_blockprod forms P_k = M_{k s + len - 1} ... M_{k s} for all blocks k in parallel, the
// chain runs over the P_k (psi(t_{ks}), chi(t_{ks})), and k_fill recovers the states inside every
// block from its first (psi) or last (chi) state, all blocks at once.

// grid (Nc, B), 256 threads, dynamic shared memory 3 tiles.  Q = T P column-major (X(i, j) at
// X[j ldm + i]).
template <typename R>
__global__ void __launch_bounds__(256) k_blockprod(ChainParams p) {
  using R2 = typename C2<R>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int k = blockIdx.x, b = blockIdx.y, d = p.d, ldm = p.ldm, N = p.N, s = p.sblk;
  const long tst = p.tile_stride;
  R2* P = reinterpret_cast<R2*>(smem_raw);
  R2* T = P + tst;
  R2* Q = T + tst;
  const R2* Mb = reinterpret_cast<const R2*>(p.M) + ((long)b * N + (long)k * s) * tst;
  const int len = min(s, N - k * s);
  for (long i = threadIdx.x; i < tst; i += blockDim.x) P[i] = Mb[i];
  for (int r = 1; r < len; ++r) {
    for (long i = threadIdx.x; i < tst; i += blockDim.x) T[i] = Mb[(long)r * tst + i];
    __syncthreads();
    // register tiles of 2 rows x 4 columns: 6 shared loads per 8 complex multiply-adds
    const int nbi = (d + 1) / 2, nbj = (d + 3) / 4;
    for (int tb = threadIdx.x; tb < nbi * nbj; tb += blockDim.x) {
      const int i0 = (tb % nbi) * 2, j0 = (tb / nbi) * 4;
      R zr[2][4], zi[2][4];
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) { zr[a][c] = R(0); zi[a][c] = R(0); }
      for (int q = 0; q < d; ++q) {
        R2 ta[2], pc[4];
#pragma unroll
        for (int a = 0; a < 2; ++a) {
          const int i = i0 + a < d ? i0 + a : d - 1;   // padded rows/columns compute a copy, not stored
          ta[a] = T[q * ldm + i];
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int j = j0 + c < d ? j0 + c : d - 1;
          pc[c] = P[j * ldm + q];
        }
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            zr[a][c] = fma(ta[a].x, pc[c].x, fma(-ta[a].y, pc[c].y, zr[a][c]));
            zi[a][c] = fma(ta[a].x, pc[c].y, fma(ta[a].y, pc[c].x, zi[a][c]));
          }
      }
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c)
          if (i0 + a < d && j0 + c < d) {
            R2 z;
            z.x = zr[a][c];
            z.y = zi[a][c];
            Q[(j0 + c) * ldm + i0 + a] = z;
          }
    }
    __syncthreads();
    R2* tmp = P;
    P = Q;
    Q = tmp;
  }
  R2* dst = reinterpret_cast<R2*>(p.Mc) + ((long)b * p.Nc + k) * tst;
  for (long i = threadIdx.x; i < tst; i += blockDim.x) dst[i] = P[i];
}

// grid (Nc, B, 2), consumer-layout threads, dynamic shared memory: the block's tiles.  z = 0: psi
// forward from psi(t_{ks}) (psi_i for k = 0), z = 1: chi backward from chi(t_{ks + len}) (chi(T) in
// FP64 for the last block); both write the FP32 staging the chain writes.
template <typename R, int JC>
__global__ void __launch_bounds__(CHAIN_MAX_THREADS) k_fill(ChainParams p) {
  using R2 = typename C2<R>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(16) R2 xs[2][64];
  const int k = blockIdx.x, b = blockIdx.y, herm = blockIdx.z, t = threadIdx.x;
  const int d = p.d, N = p.N, s = p.sblk;
  const long tst = p.tile_stride;
  const int j0 = k * s, len = min(s, N - j0);
  R2* tiles = reinterpret_cast<R2*>(smem_raw);
  const R2* Mb = reinterpret_cast<const R2*>(p.M) + ((long)b * N + j0) * tst;
  for (long i = t; i < (long)len * tst; i += blockDim.x) tiles[i] = Mb[i];
  R2* sps = reinterpret_cast<R2*>(p.stage) + (long)b * 2 * (N + 1) * d;
  R2* sch = sps + (long)(N + 1) * d;
  const double2* chin = p.chin + (long)b * (N + 1) * d;
  if (t < d) {
    R2 z;
    if (!herm) {
      if (j0 == 0) { z.x = (R)p.psi_i[t].x; z.y = (R)p.psi_i[t].y; }
      else z = sps[(long)j0 * d + t];
    } else {
      if (j0 + len == N) { z.x = (R)chin[(long)N * d + t].x; z.y = (R)chin[(long)N * d + t].y; }
      else z = sch[(long)(j0 + len) * d + t];
    }
    xs[0][t] = z;
  }
  __syncthreads();
  ChainIdx<JC> ix;
  ix.init(d, p.ldm, herm != 0);
  for (int c = 1; c < len; ++c) {   // results at j0 + c (psi) or j0 + len - c (chi)
    if (!herm) chain_mv<R, false, JC>(tiles + (long)(c - 1) * tst, xs[(c - 1) & 1], xs[c & 1], ix, d);
    else chain_mv<R, true, JC>(tiles + (long)(len - c) * tst, xs[(c - 1) & 1], xs[c & 1], ix, d);
    __syncthreads();
    if (t < d) (herm ? sch : sps)[(long)(herm ? j0 + len - c : j0 + c) * d + t] = xs[c & 1][t];
  }
}

// grid (ceil((N+2)/4), B), 128 threads: warp w of block x handles index n = 4x + w.  For n <= N it
// converts psi(t_n), chi(t_n) from the chain to FP64 (psi(t_0) = psi_i and chi(t_N) = chi(T) are
// exact), renormalises them in FP64 and forms phi_n = a_n psi(t_n) + b_n chi(t_n) (Eq. (cible));
// n = N+1 forms J and F at u in FP64.  Warp-level sums only: no block barrier.
__device__ __forceinline__ double warp_sum_d(double v) {
  for (int m = 16; m >= 1; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
  return v;
}

template <typename R>
__global__ void __launch_bounds__(128) k_phi(ChainParams p) {
  using R2 = typename C2<R>::T;
  const int lane = threadIdx.x & 31, b = blockIdx.y, d = p.d, N = p.N;
  const int n = blockIdx.x * 4 + (threadIdx.x >> 5);
  if (n > N + 1) return;   // whole warps leave
  double2* psin = p.psin + (long)b * (N + 1) * d;
  double2* chin = p.chin + (long)b * (N + 1) * d;
  const double2* psi_i = p.het ? p.psi_i + (long)b * d : p.psi_i;
  const double2* ab = p.het ? p.rt.ab + (long)b * (N + 1) : p.ab;
  const double nrm_psi_i = p.het ? p.rt.nrm[2 * b] : p.nrm_psi_i;
  const double inv_nrm_psi_i = p.het ? (nrm_psi_i > 0.0 ? 1.0 / nrm_psi_i : 0.0) : p.inv_nrm_psi_i;
  const double tau = p.het ? p.rt.tau[b] : p.tau;
  const R2* sps = reinterpret_cast<const R2*>(p.stage) + (long)b * 2 * (N + 1) * d;
  const R2* sch = sps + (long)(N + 1) * d;
  auto load_ps = [&](int m, int e) -> double2 {
    if (m == 0) return psi_i[e];
    if (p.src64) return psin[(long)m * d + e];
    const R2 z = sps[(long)m * d + e];
    return make_double2((double)z.x, (double)z.y);
  };
  auto load_cs = [&](int m, int e) -> double2 {
    if (m == N || p.src64) return chin[(long)m * d + e];
    const R2 z = sch[(long)m * d + e];
    return make_double2((double)z.x, (double)z.y);
  };
  // Norm renormalisation in FP64: the propagation is unitary, so psi(t_n) keeps the norm of psi_i
  // and chi(t_n) that of chi(T); rescaling them back removes the norm drift of FP32 propagation (a
  // no-op in exact arithmetic) and the largest relative drift is recorded.
  // reference norms: |psi_i|^2 and, for the overlap objective, |chi(T)|^2 = |psi_f|^2 come from the host;
  // the observable's chi(T) = O psi(T) differs per problem and is summed here (FP64 is scarce on this
  // GPU: no divisions, one reciprocal square root per state)
  double a = 0.0, c = 0.0, cT = p.het ? (p.nrm_chi_T < 0.0 ? -1.0 : p.rt.nrm[2 * b + 1]) : p.nrm_chi_T;
  const int m = n <= N ? n : N;
  const double* nb = p.nrm ? p.nrm + (long)b * (N + 1) * 2 : nullptr;
  if (nb) {   // squared norms left by the direct sweeps (psi(t_0) = psi_i and chi(T) are the references)
    a = m == 0 ? nrm_psi_i : nb[2 * m];
    if (cT < 0.0) cT = nb[2 * N + 1];
    c = m == N ? cT : nb[2 * m + 1];
  } else {
    for (int e = lane; e < d; e += 32) {
      const double2 x = load_ps(m, e), y = load_cs(m, e);
      a = fma(x.x, x.x, fma(x.y, x.y, a));
      c = fma(y.x, y.x, fma(y.y, y.y, c));
    }
    a = warp_sum_d(a);
    c = warp_sum_d(c);
  }
  if (cT < 0.0) {
    double t = 0.0;
    for (int e = lane; e < d; e += 32) {
      const double2 yT = chin[(long)N * d + e];
      t = fma(yT.x, yT.x, fma(yT.y, yT.y, t));
    }
    cT = warp_sum_d(t);
  }
  // relative drifts of the squared norms and the scales (1 + delta)^(-1/2), by the series
  // 1 - delta/2 + 3 delta^2/8 (truncation below 4e-13 for |delta| < 1e-4; rsqrt beyond): FP64 square
  // roots and divisions for each of the ~10^5-10^6 states of a batched step would cost more than
  // the rest of this kernel.  The drift of chi needs |psi_f|^2 or |chi(T)|^2 inverted only to FP32
  // accuracy (it multiplies a drift of ~1e-6).
  const double a0 = nrm_psi_i;
  const bool okp = a > 0.0 && a0 > 0.0, okc = c > 0.0 && cT > 0.0;
  const double dp = okp ? fma(a, inv_nrm_psi_i, -1.0) : 0.0;
  const double dc = okc ? (c - cT) * (double)(1.0f / (float)cT) : 0.0;
  auto inv_sqrt1p = [](double dl) { return fabs(dl) < 1e-4 ? fma(fma(0.375, dl, -0.5), dl, 1.0) : rsqrt(1.0 + dl); };
  const double s_psi = inv_sqrt1p(dp);
  const double s_chi = inv_sqrt1p(dc);
  if (n <= N) {
    // the drift is recorded where the propagation is longest, psi(T) and chi(t_0) (block-uniform
    // reads of one address by every state of a batch would cost more than the states themselves)
    if (lane == 0 && p.drift && okp && okc && (n == N || n == 0)) {
      const double dr = n == N ? fabs(dp) : fabs(dc);
      // non-negative doubles order as their bit patterns; read first, so that the hundreds of
      // thousands of warps of a batched launch do not all queue atomics on one address
      const unsigned long long bits = (unsigned long long)__double_as_longlong(dr);
      if (dr >= 0.0 && bits > *reinterpret_cast<volatile unsigned long long*>(p.drift)) atomicMax(p.drift, bits);
    }
    // psi_i and chi(T) are the references; psi(T) stays as propagated in psin (the J warp reads it
    // concurrently and applies the scale to its sums; chi(T) = O psi(T) was formed from it)
    const double sp = (n == 0 || n == N) ? 1.0 : s_psi;
    const double sc = n == N ? 1.0 : s_chi;
    const double2 w = ab[n];
    double2* phi = p.phi + ((long)b * (N + 1) + n) * d;
    auto put = [&](int e, double2 ps, double2 cs) {
      ps.x *= sp; ps.y *= sp;
      cs.x *= sc; cs.y *= sc;
      psin[(long)n * d + e] = ps;   // psi(t_0) = psi_i too: the chain path has not written it
      if (n < N) chin[(long)n * d + e] = cs;
      phi[e] = n == 0 ? ps : (n == N ? cs : make_double2(w.x * ps.x + w.y * cs.x, w.x * ps.y + w.y * cs.y));
    };
    if (d <= 64) {   // both elements of each lane loaded before any store: one round trip, not two
      const int e0 = lane, e1 = lane + 32;
      double2 ps0 = make_double2(0.0, 0.0), cs0 = ps0, ps1 = ps0, cs1 = ps0;
      if (e0 < d) { ps0 = load_ps(n, e0); cs0 = load_cs(n, e0); }
      if (e1 < d) { ps1 = load_ps(n, e1); cs1 = load_cs(n, e1); }
      if (e0 < d) put(e0, ps0, cs0);
      if (e1 < d) put(e1, ps1, cs1);
      return;
    }
    for (int e = lane; e < d; e += 32) put(e, load_ps(n, e), load_cs(n, e));
    return;
  }
  // J and F: <psi(T)|chi(T)> is the overlap with psi_f or <psi|O|psi>, with psi(T) renormalised (the
  // scale is applied to the sums).  Overlap objective: chi(T) = psi_f, linear in psi(T); observable:
  // chi(T) = O psi(T) was formed from the unscaled psi(T), so <psi|O|psi> takes the scale twice.
  double ovr = 0.0, ovi = 0.0;
  for (int e = lane; e < d; e += 32) {
    const double2 z = load_ps(N, e);
    const double2 y = chin[(long)N * d + e];
    ovr += z.x * y.x + z.y * y.y;
    ovi += z.x * y.y - z.y * y.x;
  }
  ovr = warp_sum_d(ovr);
  ovi = warp_sum_d(ovi);
  const double sj = p.obj == 0 ? s_psi : s_psi * s_psi;
  ovr *= sj;
  ovi *= sj;
  double pen = 0.0;
  if (p.pen)
    for (int n2 = lane; n2 < N; n2 += 32) pen += p.pen[(long)b * N + n2];
  pen = 0.5 * tau * warp_sum_d(pen);
  if (lane == 0) {
    const double F = p.obj == 0 ? ovr * ovr + ovi * ovi : ovr;
    const double J = ovr - pen;
    if (!isfinite(J) || !isfinite(F)) atomicOr(p.status, ST_NONFINITE);
    p.J[b] = J;
    p.F[b] = F;
    if (p.Jhist) p.Jhist[(long)b * p.hist_stride + p.hist_k] = J;
  }
}

}  // namespace ism
