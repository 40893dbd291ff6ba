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
#include "ism_device.cuh"

namespace ism {

struct KParams {
  int d, Nt, N, B, ldm, dpad;
  double tau, T, c0, r0, h1n, tol, rho, w;
  const int* jn;          // [N+1] step boundaries
  const double* beta;     // [N]
  const double* alpha;    // [Nt] or null
  const void* H;          // packed op data (element type R)
  const double* H0d;      // FP64 diagonal of H0 (tridiagonal and bit-flip kinds)
  double* u;              // [B][Nt]
  const double2* phi;     // [B][N+1][d]
  void* M;                // [B][N] tiles of tile_stride R2: [d cols][ldm rows], ldm odd >= d
  long tile_stride;
  void* traj;             // [B][Nt+N][G*E] (R2)  H1 psi_n(t_j) per step
  double* grad;           // [B][Nt]
  double* Jn;             // [B][N]
  double* err;            // [B][N]
  int* status;
  unsigned long long* count;   // [3]: Y applications, accumulated terms, exp sub-steps (or null)
  const double2* psin;         // [B][N+1][d] psi(t_n) (form 1)
  const double2* chin;         // [B][N+1][d] chi(t_n) (form 1)
  int form;                    // 0: literal sub-problem from phi; 1: Theorem 2 two-trajectory form
  int update;
  int max_spin;
};

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
  double2* phi;           // [B][N+1][d]
  double* J;              // [B]
  double* F;              // [B]
  double* Jhist;          // [B][hist_stride] or null
  int hist_stride, hist_k;
  int stages;             // bulk-copy ring depth per chain (2..CHAIN_MAX_STAGES)
  long tile_stride;       // R2 elements between consecutive tiles (d*ldm rounded up to even)
  int* status;
  int max_spin;
};

template <typename R> __device__ __forceinline__ R ldu_ro(const double* u, long i) { return (R)__ldg(u + i); }
template <typename R> __device__ __forceinline__ R ldu(const double* u, long i) { return (R)u[i]; }

// Work accounting: one group adds its applications of Y, accumulated series terms and exp sub-steps.
template <typename R>
__device__ __forceinline__ void count_work(unsigned long long* c, const Cheb<R>& ch, long steps, int lg) {
  if (c && lg == 0 && steps > 0) {
    atomicAdd(c + 0, (unsigned long long)(steps * ch.S * (ch.K - 1)));
    atomicAdd(c + 1, (unsigned long long)(steps * ch.S * ch.K));
    atomicAdd(c + 2, (unsigned long long)(steps * ch.S));
  }
}

// ------------------------------------------------------------------------------ k_assemble
template <typename R, class Op>
__global__ void __launch_bounds__(128) k_assemble(KParams p) {
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
    for (int i = threadIdx.x; i < 2 * Op::DP_SMEM * Op::DP_SMEM; i += blockDim.x) dst[i] = src[i];
    __syncthreads();
  }
  if (gid >= total) return;
  const int col = (int)(gid % p.dpad);
  const long bn = gid / p.dpad;
  const int n = (int)(bn % p.N), b = (int)(bn / p.N);
  const int j0 = p.jn[n], j1 = p.jn[n + 1];
  const double* ub = p.u + (long)b * p.Nt;

  double um = 0.0;
  for (int j = j0 + lg; j < j1; j += G) um = fmax(um, fabs(ub[j]));
  um = g_max<G>(um);
  Cheb<R>& ch = chs[gib];
  cheb_setup<G, R>(ch, lg, p.tau, p.c0, p.r0, p.h1n, um, p.tol, p.status);

  Op op;
  op.load(reinterpret_cast<const R*>(p.H), p.H0d, p.d, lg, smem_raw);
  op.scale(p.H0d, p.d, lg, ch);
  Vec<R, E> v, lo;
#pragma unroll
  for (int r = 0; r < E; ++r) {
    v.re[r] = (lg * E + r == col) ? R(1) : R(0);
    v.im[r] = R(0);
    lo.re[r] = R(0);
    lo.im[r] = R(0);
  }

  // controls two steps ahead in registers
  R ua = ldu_ro<R>(ub, j0), ub1 = j0 + 1 < j1 ? ldu_ro<R>(ub, j0 + 1) : R(0);
  for (int j = j0; j < j1; ++j) {
    const R uj = ua;
    ua = ub1;
    if (j + 2 < j1) ub1 = ldu_ro<R>(ub, j + 2);
    op.set_u(uj, ch, lg);
    cheb_step<false, COMP>(v, lo, op, ch);
  }
  if (col < p.d) {
    count_work<R>(p.count, ch, j1 - j0, lg);
    double sn, cs;   // global phase exp(-i c (t_{n+1} - t_n)) of the whole sub-interval, FP64
    sincos(p.c0 * p.tau * (double)(j1 - j0), &sn, &cs);
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

// ------------------------------------------------------------------------------ k_subinterval
// One group per (problem, n).  Sequential part per step: the propagation (forward, then adjoint) and
// an FP32 group reduction; the FP64 gradient, Err and ascent step are done afterwards with the lanes
// working on different steps.  The trajectory slot of step j (H1 psi_n(t_j), consumed by the backward
// sweep at step j) is reused to hold the gradient term Im<delta_j|H1 psi_j> for that final pass.
template <typename R, class Op>
__global__ void __launch_bounds__(128) k_subinterval(KParams p) {
  constexpr int G = Op::G, E = Op::E, GPB = 128 / G, GE = G * E;
  constexpr bool COMP = sizeof(R) == 4;
  using R2 = typename C2<R>::T;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ Cheb<R> chs[GPB];
  const int lg = threadIdx.x % G, gib = threadIdx.x / G;
  const long gid0 = (long)blockIdx.x * GPB + gib;
  const long total = (long)p.B * p.N;
  if (Op::G * Op::E == Op::DP_SMEM) {
    const R* src = reinterpret_cast<const R*>(p.H);
    R* dst = reinterpret_cast<R*>(smem_raw);
    for (int i = threadIdx.x; i < 2 * Op::DP_SMEM * Op::DP_SMEM; i += blockDim.x) dst[i] = src[i];
    __syncthreads();
  }
  // warps whose groups are all past the end leave; partially valid warps keep every lane running
  const long warp_first = ((long)blockIdx.x * GPB + (threadIdx.x / 32) * (32 / G));
  if (warp_first >= total) return;
  const bool valid = gid0 < total;
  const long gid = valid ? gid0 : total - 1;
  const int n = (int)(gid % p.N), b = (int)(gid / p.N);
  const int j0 = p.jn[n], j1 = p.jn[n + 1], ns = j1 - j0;
  const int nsw = warp_max_i(ns);
  double* ub = p.u + (long)b * p.Nt;
  const double beta = p.beta[n];

  double um = 0.0;
  for (int j = j0 + lg; j < j1; j += G) um = fmax(um, fabs(ub[j]));
  um = g_max<G>(um);
  Cheb<R>& ch = chs[gib];
  cheb_setup<G, R>(ch, lg, p.tau, p.c0, p.r0, p.h1n, um, p.tol, p.status);

  Op op;
  op.load(reinterpret_cast<const R*>(p.H), p.H0d, p.d, lg, smem_raw);
  op.scale(p.H0d, p.d, lg, ch);
  // Propagation here omits the global phase exp(-i c tau) of each step.  Over the sub-interval it
  // multiplies psi_n(t_{n+1}) by exp(-i Phi), Phi = c (t_{n+1} - t_n), and every gradient term
  // <chi_n|H1|psi_n>(t_j) by the same exp(-i Phi) (chi_n carries exp(+i c (t_{n+1} - t_j)), psi_n
  // exp(-i c (t_j - t_n))); both are applied once, in FP64.
  double sPhi, cPhi;
  sincos(p.c0 * p.tau * (double)ns, &sPhi, &cPhi);

  // form 0: psi_n(t_n) = phi_n (Eq. (dirpara)), adjoint from phi_{n+1};
  // form 1 (phi = phi^u, first local step): psi from psi(t_n) and chi from chi(t_{n+1}), the two
  // trajectories of which psi_n, chi_n are combinations (proof of Theorem 2); no cancellation.
  const long off_n = ((long)b * (p.N + 1) + n) * p.d;
  const double2* phn = (p.form ? p.psin : p.phi) + off_n;
  const double2* phn1 = (p.form ? p.chin : p.phi) + off_n + p.d;
  Vec<R, E> v, lo;
#pragma unroll
  for (int r = 0; r < E; ++r) {
    int e = lg * E + r;
    double2 z = e < p.d ? phn[e] : make_double2(0.0, 0.0);
    v.re[r] = (R)z.x;
    v.im[r] = (R)z.y;
    lo.re[r] = COMP ? (R)(z.x - (double)v.re[r]) : R(0);
    lo.im[r] = COMP ? (R)(z.y - (double)v.im[r]) : R(0);
  }
  R2* tr0 = reinterpret_cast<R2*>(p.traj) + ((long)b * (p.Nt + p.N) + j0 + n) * GE;   // slot s at tr0 + s*GE
  R2* tr = tr0 + lg * E;

  // ---- forward sweep: store H1 psi_j, then psi_{j+1} = U_j psi_j
  {
    R ua = ldu<R>(ub, j0), ub1 = ns > 1 ? ldu<R>(ub, j0 + 1) : ua;
    for (int s = 0; s < nsw; ++s) {
      const bool act = s < ns;
      const R uj = ua;
      ua = ub1;
      if (s + 2 < ns) ub1 = ldu<R>(ub, j0 + s + 2);
      Vec<R, E> hv;
      op.h1(v, hv);
      if (act && valid) {
#pragma unroll
        for (int r = 0; r < E; ++r) { R2 z; z.x = hv.re[r]; z.y = hv.im[r]; tr[(long)s * GE + r] = z; }
      }
      Vec<R, E> w = v, wl = lo;
      op.set_u(uj, ch, lg);
      cheb_step<false, COMP>(w, wl, op, ch);
      if (act) { v = w; lo = wl; }
    }
  }
  // end point: H1 psi_n(t_{n+1}) stays in registers
  Vec<R, E> hend;
  op.h1(v, hend);

  // ---- terminal residual delta = phi_{n+1} - psi_n(t_{n+1}) in FP64 (its norm gives J_n).  Form 0
  // propagates delta backward; form 1 propagates chi from chi(t_{n+1}) and takes delta from the
  // chain, delta = (chi - psi)(t_{n+1}) / beta_n.
  double nrm = 0.0;
  Vec<R, E> dl;
#pragma unroll
  for (int r = 0; r < E; ++r) {
    int e = lg * E + r;
    double2 z = e < p.d ? phn1[e] : make_double2(0.0, 0.0);
    double dr, di;
    if (!p.form) {
      double pr, pi;
      phase_rotate(cPhi, sPhi, false, (double)v.re[r] + (double)lo.re[r], (double)v.im[r] + (double)lo.im[r], pr, pi);
      dr = z.x - pr;
      di = z.y - pi;
      dl.re[r] = (R)dr;
      dl.im[r] = (R)di;
    } else {
      double2 ps = e < p.d ? p.psin[off_n + p.d + e] : make_double2(0.0, 0.0);
      dr = (z.x - ps.x) / beta;
      di = (z.y - ps.y) / beta;
      dl.re[r] = (R)z.x;
      dl.im[r] = (R)z.y;
    }
    if (e >= p.d) { dr = 0.0; di = 0.0; }
    nrm += dr * dr + di * di;
  }
  nrm = g_sum<G>(nrm);

  // z = <a|h> over the group, FP32 products, both parts (the phase exp(-i Phi) is applied later)
  auto zdot = [&](const Vec<R, E>& a, const Vec<R, E>& h, R& zr, R& zi) {
    R xr = R(0), xi = R(0);
#pragma unroll
    for (int r = 0; r < E; ++r) {
      xr = fma(a.re[r], h.re[r], fma(a.im[r], h.im[r], xr));
      xi = fma(a.re[r], h.im[r], fma(-a.im[r], h.re[r], xi));
    }
    zr = g_sum<G>(xr);
    zi = g_sum<G>(xi);
  };
  {
    R zr, zi;
    zdot(dl, hend, zr, zi);
    if (lg == 0 && valid) { R2 z; z.x = zr; z.y = zi; tr0[(long)ns * GE] = z; }
  }

  // ---- backward sweep: delta_j = U_j^H delta_{j+1}; gradient term of step j into slot j
  {
    const int top = ns - 1;
    Vec<R, E> h0, h1v;   // slots s and s-1, prefetched
    auto ldslot = [&](int s, Vec<R, E>& h) {
#pragma unroll
      for (int r = 0; r < E; ++r) { R2 z = tr[(long)s * GE + r]; h.re[r] = z.x; h.im[r] = z.y; }
    };
    ldslot(top, h0);
    ldslot(top > 0 ? top - 1 : top, h1v);
    R ua = ldu<R>(ub, j0 + top), ub1 = ldu<R>(ub, j0 + (top > 0 ? top - 1 : top));
    for (int s = nsw - 1; s >= 0; --s) {
      const bool act = s < ns;
      Vec<R, E> hc = h0;
      const R uj = ua;
      if (act) {
        h0 = h1v;
        ua = ub1;
        if (s - 2 >= 0) { ldslot(s - 2, h1v); ub1 = ldu<R>(ub, j0 + s - 2); }
      }
      Vec<R, E> w = dl;
      op.set_u(uj, ch, lg);
      cheb_step<true>(w, op, ch);
      if (act) dl = w;
      R zr, zi;
      zdot(dl, hc, zr, zi);
      if (act && lg == 0 && valid) { R2 z; z.x = zr; z.y = zi; tr0[(long)s * GE] = z; }
    }
  }
  __syncwarp();

  // ---- FP64 pass over the steps: gradient, Err, ascent step, penalty of J_n
  const double ht = 0.5 * p.tau * p.w / (p.form ? beta : 1.0);
  const double tb = p.tau / beta;
  const double step = p.rho * beta / p.tau;
  double* gb = p.grad + (long)b * p.Nt;
  double err = 0.0, pen = 0.0;
  for (int s = lg; s < ns; s += G) {
    const int j = j0 + s;
    const double uj = ub[j];
    const double al = p.alpha ? p.alpha[j] : 0.0;
    const R2 za = tr0[(long)s * GE], zb = tr0[(long)(s + 1) * GE];
    // Im(exp(-i Phi) z) for the two ends of step j
    const double Ia = cPhi * (double)za.y - sPhi * (double)za.x;
    const double Ib = cPhi * (double)zb.y - sPhi * (double)zb.x;
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
  const double Jn = p.w * (-0.5 * nrm) - 0.5 * tb * pen;
  if (lg == 0 && valid) {
    if (p.Jn) p.Jn[gid] = Jn;
    if (p.err) p.err[gid] = err;
  }
  if (valid) count_work<R>(p.count, ch, 2L * ns, lg);   // forward U and backward U^H sweeps
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
// The chain is a sequence of 2N small dependent matvecs: latency, not bandwidth.  The tiles M_n (left
// in L2 by the assembly) stream into a ring of NS shared-memory stages by TMA bulk copies issued up to
// NS - 1 matvecs ahead; thread 0 alone waits on a stage's mbarrier (bounded), and one block barrier
// per matvec publishes both the tile and the previous result.  256 threads: thread (i = t/4, q = t%4)
// owns output row i and the columns k = q (mod 4); two shuffles finish each row.
constexpr int CHAIN_MAX_STAGES = 16;

template <typename R>
__device__ __forceinline__ void chain_mv(const typename C2<R>::T* Ms, const typename C2<R>::T* x,
                                         typename C2<R>::T* y, int d, int ldm, bool herm) {
  using R2 = typename C2<R>::T;
  const int i = threadIdx.x >> 2, q = threadIdx.x & 3;
  R ar0 = R(0), ai0 = R(0), ar1 = R(0), ai1 = R(0);
  if (i < d) {
#pragma unroll 4
    for (int k = q; k < d; k += 8) {
      {
        const R2 m = herm ? Ms[i * ldm + k] : Ms[k * ldm + i];
        const R2 xv = x[k];
        if (!herm) { ar0 = fma(m.x, xv.x, fma(-m.y, xv.y, ar0)); ai0 = fma(m.x, xv.y, fma(m.y, xv.x, ai0)); }
        else { ar0 = fma(m.x, xv.x, fma(m.y, xv.y, ar0)); ai0 = fma(m.x, xv.y, fma(-m.y, xv.x, ai0)); }
      }
      const int k2 = k + 4;
      if (k2 < d) {
        const R2 m = herm ? Ms[i * ldm + k2] : Ms[k2 * ldm + i];
        const R2 xv = x[k2];
        if (!herm) { ar1 = fma(m.x, xv.x, fma(-m.y, xv.y, ar1)); ai1 = fma(m.x, xv.y, fma(m.y, xv.x, ai1)); }
        else { ar1 = fma(m.x, xv.x, fma(m.y, xv.y, ar1)); ai1 = fma(m.x, xv.y, fma(-m.y, xv.x, ai1)); }
      }
    }
  }
  R ar = ar0 + ar1, ai = ai0 + ai1;
  ar += __shfl_xor_sync(0xffffffffu, ar, 1);
  ai += __shfl_xor_sync(0xffffffffu, ai, 1);
  ar += __shfl_xor_sync(0xffffffffu, ar, 2);
  ai += __shfl_xor_sync(0xffffffffu, ai, 2);
  if (q == 0 && i < d) { R2 z; z.x = ar; z.y = ai; y[i] = z; }
}

// The ring: use m (0..U-1) of the chain(s) this CTA runs reads tile tile_of(m) from stage m % NS.
template <typename R>
struct ChainRing {
  using R2 = typename C2<R>::T;
  R2* stages;
  uint64_t* bars;
  const R2* Mb;
  long tst;
  unsigned bytes;
  int NS, U, N, first;   // tile_of(m): first == 0 -> m < N ? m : 2N-1-m; first == 1 -> N-1-m
  __device__ int tile_of(int m) const { return first == 1 ? N - 1 - m : (m < N ? m : 2 * N - 1 - m); }
  __device__ void issue(int m) const {   // thread 0
    const int st = m % NS;
    fence_proxy_async();
    bulk_load(stages + st * tst, Mb + (long)tile_of(m) * tst, bytes, &bars[st]);
  }
  __device__ const R2* tile(int m) const { return stages + (m % NS) * tst; }
};

// One chain of N matvecs over uses m0 .. m0+N-1 of the ring; x_0 in xs[0]; writes the N results (FP64)
// into out[idx(m)*d] with idx = m - m0 + 1 (psi) or N - 1 - (m - m0) (chi).  Returns false (uniformly)
// if a tile did not arrive; the copies still in flight have then been drained.
template <typename R, bool HERM>
__device__ bool run_chain(const ChainRing<R>& ring, int m0, int N, int d, int ldm, typename C2<R>::T (*xs)[64],
                          double2* out, int* fail, int* status, int max_spin) {
  using R2 = typename C2<R>::T;
  const int t = threadIdx.x;
  for (int c = 0; c <= N; ++c) {
    const int m = m0 + c;
    if (t == 0 && c < N) {
      if (!mbar_wait(&ring.bars[m % ring.NS], (unsigned)((m / ring.NS) & 1), max_spin)) {
        for (int q = m; q < ring.U && q < m + ring.NS; ++q)
          mbar_wait(&ring.bars[q % ring.NS], (unsigned)((q / ring.NS) & 1), max_spin);
        atomicOr(status, ST_TIMEOUT);
        *fail = 1;
      }
    }
    __syncthreads();   // tile m present; result of matvec c-1 visible
    if (*fail) return false;
    if (c >= 1) {
      // the stage of use m-1 has been read by everyone: refill it NS uses ahead
      if (t == 0 && m - 1 + ring.NS < ring.U) ring.issue(m - 1 + ring.NS);
      const int idx = HERM ? N - c : c;
      if (t < d) { const R2 z = xs[c & 1][t]; out[(long)idx * d + t] = make_double2((double)z.x, (double)z.y); }
    }
    if (c < N) chain_mv<R>(ring.tile(m), xs[c & 1], xs[(c + 1) & 1], d, ldm, HERM);
  }
  __syncthreads();   // the last stored state is read by other threads next
  return true;
}

// grid (nchains, B), 256 threads, dynamic shared memory NS tiles.  nchains = 2 (overlap objective):
// CTA 0 runs the psi chain, CTA 1 the chi chain from psi_f, concurrently.  nchains = 1 (observable):
// one CTA runs the psi chain, forms chi(T) = O psi(T) in FP64 and runs the chi chain, all from one ring.
// Intermediate states and J follow in k_phi.
template <typename R>
__global__ void __launch_bounds__(256) k_chain(ChainParams p) {
  using R2 = typename C2<R>::T;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bars[CHAIN_MAX_STAGES];
  __shared__ __align__(16) R2 xs[2][64];
  __shared__ double2 vd[64];
  __shared__ int fail;
  const int b = blockIdx.y, t = threadIdx.x, d = p.d, N = p.N;
  double2* psin = p.psin + (long)b * (N + 1) * d;
  double2* chin = p.chin + (long)b * (N + 1) * d;
  const bool single = gridDim.x == 1;
  const bool do_psi = single || blockIdx.x == 0;
  const bool do_chi = single || blockIdx.x == 1;
  ChainRing<R> ring;
  ring.stages = reinterpret_cast<R2*>(smem_raw);
  ring.bars = bars;
  ring.Mb = reinterpret_cast<const R2*>(p.M) + (long)b * N * p.tile_stride;
  ring.tst = p.tile_stride;
  ring.bytes = (unsigned)(p.tile_stride * sizeof(R2));
  ring.NS = p.stages;
  ring.N = N;
  ring.U = single ? 2 * N : N;
  ring.first = (!single && blockIdx.x == 1) ? 1 : 0;
  if (t == 0) {
    fail = 0;
    for (int i = 0; i < ring.NS; ++i) mbar_init(&bars[i], 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (t == 0)
    for (int m = 0; m < ring.NS && m < ring.U; ++m) ring.issue(m);

  int m0 = 0;
  if (do_psi) {
    if (t < d) { const double2 z = p.psi_i[t]; R2 r; r.x = (R)z.x; r.y = (R)z.y; xs[0][t] = r; psin[t] = z; }
    if (!run_chain<R, false>(ring, m0, N, d, p.ldm, xs, psin, &fail, p.status, p.max_spin)) return;
    m0 += N;
  }
  if (do_chi) {
    if (p.obj == 0) {
      if (t < d) vd[t] = p.psi_f[t];
    } else {   // chi(T) = O psi(T), FP64, thread (i, q) sums k = q (mod 4)
      const int i = t >> 2, q = t & 3;
      double sr = 0.0, si = 0.0;
      if (i < d)
        for (int k = q; k < d; k += 4) {
          const double o = p.O[i * d + k];
          const double2 v = psin[(long)N * d + k];
          sr += o * v.x;
          si += o * v.y;
        }
      sr += __shfl_xor_sync(0xffffffffu, sr, 1);
      si += __shfl_xor_sync(0xffffffffu, si, 1);
      sr += __shfl_xor_sync(0xffffffffu, sr, 2);
      si += __shfl_xor_sync(0xffffffffu, si, 2);
      if (q == 0 && i < d) vd[i] = make_double2(sr, si);
    }
    __syncthreads();
    if (t < d) { const double2 z = vd[t]; R2 r; r.x = (R)z.x; r.y = (R)z.y; xs[0][t] = r; chin[(long)N * d + t] = z; }
    if (!run_chain<R, true>(ring, m0, N, d, p.ldm, xs, chin, &fail, p.status, p.max_spin)) return;
  }
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

// grid B, 256 threads: J and F at u (FP64) and the intermediate states (Eq. (cible)), with
// phi_0 = psi_i and phi_N = chi(T) exactly.
template <int V = 0>
__global__ void __launch_bounds__(1024) k_phi(ChainParams p) {
  __shared__ double red[32];
  const int b = blockIdx.x, t = threadIdx.x, d = p.d, N = p.N;
  const double2* psin = p.psin + (long)b * (N + 1) * d;
  const double2* chin = p.chin + (long)b * (N + 1) * d;
  double ovr = 0.0, ovi = 0.0;
  for (int i = t; i < d; i += blockDim.x) {
    const double2 a = psin[(long)N * d + i], c = chin[(long)N * d + i];
    ovr += a.x * c.x + a.y * c.y;
    ovi += a.x * c.y - a.y * c.x;
  }
  ovr = block_sum(ovr, red);
  ovi = block_sum(ovi, red);
  double pen = 0.0;
  if (p.alpha) {
    const double* ub = p.u + (long)b * p.Nt;
    for (int j = t; j < p.Nt; j += blockDim.x) pen += p.alpha[j] * ub[j] * ub[j];
  }
  pen = 0.5 * p.tau * block_sum(pen, red);
  if (t == 0) {
    const double F = p.obj == 0 ? ovr * ovr + ovi * ovi : ovr;
    const double J = ovr - pen;
    if (!isfinite(J) || !isfinite(F)) atomicOr(p.status, ST_NONFINITE);
    p.J[b] = J;
    p.F[b] = F;
    if (p.Jhist) p.Jhist[(long)b * p.hist_stride + p.hist_k] = J;
  }
  double2* phi = p.phi + (long)b * (N + 1) * d;
  for (long i = t; i < (long)(N + 1) * d; i += blockDim.x) {
    const int n = (int)(i / d);
    const double2 w = p.ab[n];
    const double a = w.x, c = w.y;
    const double2 ps = psin[i], cs = chin[i];
    double2 z;
    if (n == 0) z = ps;
    else if (n == N) z = cs;
    else z = make_double2(a * ps.x + c * cs.x, a * ps.y + c * cs.y);
    phi[i] = z;
  }
}

}  // namespace ism
