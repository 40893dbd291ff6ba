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
  double* u;              // [B][Nt]
  const double2* phi;     // [B][N+1][d]
  void* M;                // [B][N][d cols][ldm rows] (R2)
  void* traj;             // [B][Nt+N][G*E] (R2)  H1 psi_n(t_j) per step
  double* grad;           // [B][Nt]
  double* Jn;             // [B][N]
  double* err;            // [B][N]
  int* status;
  unsigned long long* count;   // [3]: Y applications, accumulated terms, exp sub-steps (or null)
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
  double2* psin;          // [B][N+1][d]
  double2* chin;          // [B][N+1][d]
  double2* phi;           // [B][N+1][d]
  double* J;              // [B]
  double* F;              // [B]
  double* Jhist;          // [B][hist_stride] or null
  int hist_stride, hist_k;
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
  op.load(reinterpret_cast<const R*>(p.H), p.d, lg, smem_raw);
  Vec<R, E> v;
#pragma unroll
  for (int r = 0; r < E; ++r) { v.re[r] = (lg * E + r == col) ? R(1) : R(0); v.im[r] = R(0); }

  R un = ldu_ro<R>(ub, j0);
  for (int j = j0; j < j1; ++j) {
    const R uj = un;
    if (j + 1 < j1) un = ldu_ro<R>(ub, j + 1);
    op.set_u(uj, ch, lg);
    cheb_step<false>(v, op, ch);
  }
  if (col < p.d) {
    count_work<R>(p.count, ch, j1 - j0, lg);
    R2* M = reinterpret_cast<R2*>(p.M) + (bn * p.d + col) * (long)p.ldm;
#pragma unroll
    for (int r = 0; r < E; ++r) {
      int e = lg * E + r;
      if (e < p.d) { R2 z; z.x = v.re[r]; z.y = v.im[r]; M[e] = z; }
    }
  }
}

// ------------------------------------------------------------------------------ k_subinterval
template <typename R, class Op>
__global__ void __launch_bounds__(128) k_subinterval(KParams p) {
  constexpr int G = Op::G, E = Op::E, GPB = 128 / G, GE = G * E;
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
  op.load(reinterpret_cast<const R*>(p.H), p.d, lg, smem_raw);

  // psi_n(t_n) = phi_n (FP64 -> R)
  const double2* phn = p.phi + ((long)b * (p.N + 1) + n) * p.d;
  const double2* phn1 = phn + p.d;
  Vec<R, E> v;
#pragma unroll
  for (int r = 0; r < E; ++r) {
    int e = lg * E + r;
    double2 z = e < p.d ? phn[e] : make_double2(0.0, 0.0);
    v.re[r] = (R)z.x;
    v.im[r] = (R)z.y;
  }
  R2* tr = reinterpret_cast<R2*>(p.traj) + ((long)b * (p.Nt + p.N) + j0 + n) * GE + lg * E;

  // ---- forward sweep: store H1 psi_j, then psi_{j+1} = U_j psi_j
  R un = ldu<R>(ub, j0);
  for (int s = 0; s < nsw; ++s) {
    const bool act = s < ns;
    const R uj = un;
    if (s + 1 < ns) un = ldu<R>(ub, j0 + s + 1);
    Vec<R, E> hv;
    op.h1(v, hv);
    if (act && valid) {
#pragma unroll
      for (int r = 0; r < E; ++r) { R2 z; z.x = hv.re[r]; z.y = hv.im[r]; tr[(long)s * GE + r] = z; }
    }
    Vec<R, E> w = v;
    op.set_u(uj, ch, lg);
    cheb_step<false>(w, op, ch);
    if (act) v = w;
  }
  // end point: H1 psi_n(t_{n+1}) stays in registers
  Vec<R, E> hend;
  op.h1(v, hend);

  // ---- terminal residual delta = phi_{n+1} - psi_n(t_{n+1}) in FP64; J_n
  double nrm = 0.0;
  Vec<R, E> dl;
#pragma unroll
  for (int r = 0; r < E; ++r) {
    int e = lg * E + r;
    double2 z = e < p.d ? phn1[e] : make_double2(0.0, 0.0);
    double dr = z.x - (double)v.re[r], di = z.y - (double)v.im[r];
    if (e >= p.d) { dr = 0.0; di = 0.0; }
    nrm += dr * dr + di * di;
    dl.re[r] = (R)dr;
    dl.im[r] = (R)di;
  }
  nrm = g_sum<G>(nrm);
  double pen = 0.0;
  if (p.alpha) {
    for (int j = j0 + lg; j < j1; j += G) pen += p.alpha[j] * ub[j] * ub[j];
    pen = g_sum<G>(pen);
  }
  const double Jn = p.w * (-0.5 * nrm) - 0.5 * p.tau * pen / beta;

  // Im<delta|H1 psi>: the chi-part of Im<chi_n|H1|psi_n> with chi_n = psi_n + delta (Im<psi|H1|psi> = 0)
  auto imdot = [&](const Vec<R, E>& a, const Vec<R, E>& h) -> R {
    R acc = R(0);
#pragma unroll
    for (int r = 0; r < E; ++r) acc = fma(a.re[r], h.im[r], fma(-a.im[r], h.re[r], acc));
    return g_sum<G>(acc);
  };
  double Inext = (double)imdot(dl, hend);

  // ---- backward sweep: delta_j = U_j^H delta_{j+1}, gradient terms, optional ascent step
  const double ht = 0.5 * p.tau * p.w;
  const double step = p.rho * beta / p.tau;
  double err = 0.0;
  double* gb = p.grad + (long)b * p.Nt;
  Vec<R, E> hn;
  {
    const int s0 = ns - 1;
#pragma unroll
    for (int r = 0; r < E; ++r) { R2 z = tr[(long)s0 * GE + r]; hn.re[r] = z.x; hn.im[r] = z.y; }
  }
  for (int s = nsw - 1; s >= 0; --s) {
    const bool act = s < ns;
    const int sc = act ? s : ns - 1;
    const int j = j0 + sc;
    const double ujd = ub[j];
    Vec<R, E> hc = hn;
    if (s - 1 >= 0 && s - 1 < ns) {
#pragma unroll
      for (int r = 0; r < E; ++r) { R2 z = tr[(long)(s - 1) * GE + r]; hn.re[r] = z.x; hn.im[r] = z.y; }
    }
    Vec<R, E> w = dl;
    op.set_u((R)ujd, ch, lg);
    cheb_step<true>(w, op, ch);
    if (act) dl = w;
    const double I = (double)imdot(dl, hc);
    if (act) {
      const double al = p.alpha ? p.alpha[j] : 0.0;
      const double g = ht * (I + Inext) - p.tau * (al / beta) * ujd;
      Inext = I;
      err += fabs(g);
      if (lg == 0 && valid) {
        gb[j] = g;
        if (p.update) ub[j] = ujd + step * g;
      }
    }
  }
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

template <typename R>
__device__ __forceinline__ void chain_matvec(const typename C2<R>::T* Ms, const typename C2<R>::T* x,
                                             typename C2<R>::T* y, int d, int ldm, bool herm) {
  // thread (i = t/4, q = t%4): y_i = sum over k = q mod 4 of M[i][k] x_k (M x) or conj(M[k][i]) x_k (M^H x)
  using R2 = typename C2<R>::T;
  const int t = threadIdx.x, i = t >> 2, q = t & 3;
  R ar = R(0), ai = R(0);
  if (i < d) {
    for (int k = q; k < d; k += 4) {
      R2 m = herm ? Ms[i * ldm + k] : Ms[k * ldm + i];
      R2 xv = x[k];
      if (!herm) {
        ar = fma(m.x, xv.x, fma(-m.y, xv.y, ar));
        ai = fma(m.x, xv.y, fma(m.y, xv.x, ai));
      } else {
        ar = fma(m.x, xv.x, fma(m.y, xv.y, ar));
        ai = fma(m.x, xv.y, fma(-m.y, xv.x, ai));
      }
    }
  }
  ar += __shfl_xor_sync(0xffffffffu, ar, 1);
  ai += __shfl_xor_sync(0xffffffffu, ai, 1);
  ar += __shfl_xor_sync(0xffffffffu, ar, 2);
  ai += __shfl_xor_sync(0xffffffffu, ai, 2);
  if (q == 0 && i < d) { R2 z; z.x = ar; z.y = ai; y[i] = z; }
}

__device__ inline double block_sum256(double v, double* red) {
  for (int m = 16; m >= 1; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
  return s;
}

// blockDim = 256; dynamic shared memory: 2 M tiles (R2 d*ldm each) | 2 vectors (R2 64) | FP64 work.
template <typename R>
__global__ void __launch_bounds__(256) k_chain(ChainParams p) {
  using R2 = typename C2<R>::T;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bars[2];
  __shared__ double red[8];
  __shared__ double2 vd[64];        // FP64 vector work space (psi(T), chi(T))
  const int b = blockIdx.x, t = threadIdx.x, d = p.d, N = p.N;
  const long tile = (long)d * p.ldm;
  const unsigned tbytes = (unsigned)(tile * sizeof(R2));
  R2* Mbuf[2] = {reinterpret_cast<R2*>(smem_raw), reinterpret_cast<R2*>(smem_raw) + tile};
  R2* xv[2] = {Mbuf[1] + tile, Mbuf[1] + tile + 64};
  const R2* Mg = reinterpret_cast<const R2*>(p.M) + (long)b * N * tile;
  double2* psin = p.psin + (long)b * (N + 1) * d;
  double2* chin = p.chin + (long)b * (N + 1) * d;
  bool ok = true;

  if (t == 0) { mbar_init(&bars[0], 1); mbar_init(&bars[1], 1); fence_mbar_init(); }
  __syncthreads();
  unsigned ph[2] = {0u, 0u};

  // ---- psi chain: psi(t_0) = psi_i, psi(t_{n+1}) = M_n psi(t_n)
  if (t == 0) bulk_load(Mbuf[0], Mg, tbytes, &bars[0]);
  if (t < d) { double2 z = p.psi_i[t]; R2 r; r.x = (R)z.x; r.y = (R)z.y; xv[0][t] = r; psin[t] = z; }
  __syncthreads();
  for (int n = 0; n < N; ++n) {
    const int cb = n & 1;
    const bool pre = n + 1 < N;
    if (t == 0 && pre) { fence_proxy_async(); bulk_load(Mbuf[cb ^ 1], Mg + (n + 1) * tile, tbytes, &bars[cb ^ 1]); }
    ok = mbar_wait(&bars[cb], ph[cb], p.max_spin);
    if (__syncthreads_or(!ok)) {   // a tile never arrived: drain what is in flight, report, leave
      if (t == 0) {
        mbar_wait(&bars[cb], ph[cb], p.max_spin);
        if (pre) mbar_wait(&bars[cb ^ 1], ph[cb ^ 1], p.max_spin);
        atomicOr(p.status, ST_TIMEOUT);
      }
      return;
    }
    ph[cb] ^= 1u;
    chain_matvec<R>(Mbuf[cb], xv[n & 1], xv[(n + 1) & 1], d, p.ldm, false);
    __syncthreads();
    if (t < d) { R2 z = xv[(n + 1) & 1][t]; psin[(long)(n + 1) * d + t] = make_double2((double)z.x, (double)z.y); }
  }
  // ---- terminal adjoint chi(T) and objective (FP64)
  if (t < d) vd[t] = psin[(long)N * d + t];
  __syncthreads();
  double2 chiT = make_double2(0.0, 0.0);
  if (t < d) {
    if (p.obj == 0) {
      chiT = p.psi_f[t];
    } else {
      double sr = 0.0, si = 0.0;
      for (int k = 0; k < d; ++k) { double o = p.O[t * d + k]; sr += o * vd[k].x; si += o * vd[k].y; }
      chiT = make_double2(sr, si);
    }
  }
  // <psi(T)|chi(T)> (overlap with psi_f, or <psi|O|psi>)
  double ovr = 0.0, ovi = 0.0;
  if (t < d) { double2 a = vd[t]; ovr = a.x * chiT.x + a.y * chiT.y; ovi = a.x * chiT.y - a.y * chiT.x; }
  ovr = block_sum256(ovr, red);
  ovi = block_sum256(ovi, red);
  double pen = 0.0;
  if (p.alpha) {
    const double* ub = p.u + (long)b * p.Nt;
    for (int j = t; j < p.Nt; j += blockDim.x) pen += p.alpha[j] * ub[j] * ub[j];
  }
  pen = 0.5 * p.tau * block_sum256(pen, red);
  if (t == 0) {
    double F = p.obj == 0 ? ovr * ovr + ovi * ovi : ovr;
    double J = ovr - pen;
    if (!isfinite(J) || !isfinite(F)) atomicOr(p.status, ST_NONFINITE);
    p.J[b] = J;
    p.F[b] = F;
    if (p.Jhist) p.Jhist[(long)b * p.hist_stride + p.hist_k] = J;
  }
  __syncthreads();
  // ---- chi chain: chi(t_N) = chi(T), chi(t_n) = M_n^H chi(t_{n+1})
  if (t == 0) { fence_proxy_async(); bulk_load(Mbuf[0], Mg + (long)(N - 1) * tile, tbytes, &bars[0]); }
  // the psi pass consumed phases as it went; restart both barriers' parities from their state
  if (t < d) { R2 r; r.x = (R)chiT.x; r.y = (R)chiT.y; xv[0][t] = r; chin[(long)N * d + t] = chiT; }
  __syncthreads();
  int cnt = 0;
  for (int n = N - 1; n >= 0; --n, ++cnt) {
    const int cb = cnt & 1;
    const bool pre = n - 1 >= 0;
    if (t == 0 && pre) { fence_proxy_async(); bulk_load(Mbuf[cb ^ 1], Mg + (long)(n - 1) * tile, tbytes, &bars[cb ^ 1]); }
    ok = mbar_wait(&bars[cb], ph[cb], p.max_spin);
    if (__syncthreads_or(!ok)) {
      if (t == 0) {
        mbar_wait(&bars[cb], ph[cb], p.max_spin);
        if (pre) mbar_wait(&bars[cb ^ 1], ph[cb ^ 1], p.max_spin);
        atomicOr(p.status, ST_TIMEOUT);
      }
      return;
    }
    ph[cb] ^= 1u;
    chain_matvec<R>(Mbuf[cb], xv[cnt & 1], xv[(cnt + 1) & 1], d, p.ldm, true);
    __syncthreads();
    if (t < d) { R2 z = xv[(cnt + 1) & 1][t]; chin[(long)n * d + t] = make_double2((double)z.x, (double)z.y); }
  }
  __syncthreads();
  // ---- intermediate states (Eq. (cible)), FP64: phi_0 = psi_i, phi_N = chi(T) exactly
  double2* phi = p.phi + (long)b * (N + 1) * d;
  for (long i = t; i < (long)(N + 1) * d; i += blockDim.x) {
    const int n = (int)(i / d);
    const double tn = p.jn[n] * p.tau;
    const double a = (p.T - tn) / p.T, c = tn / p.T;
    double2 ps = psin[i], cs = chin[i];
    double2 z;
    if (n == 0) z = ps;
    else if (n == N) z = cs;
    else z = make_double2(a * ps.x + c * cs.x, a * ps.y + c * cs.y);
    phi[i] = z;
  }
}

}  // namespace ism
