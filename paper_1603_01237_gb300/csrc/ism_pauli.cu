// ism_pauli.cu -- several controls on a Pauli structure (the five-spin example of Sec. 4, written in
// Liouville space): H(u) = diag(H0) + sum_c u_c H_c, H_c = sum_b (ax[c][b] X_b + ay[c][b] Y_b) on
// d = 2^q basis states (bit b of the index; Pauli Y = [[0, -i], [i, 0]], so (Y_b v)[e] =
// i s_b(e) v[e ^ 2^b] with s_b(e) = +1 when bit b of e is set, -1 otherwise).  d = 128 .. 1024, one
// state per CTA of d/4 threads, element e = 4 t + r of thread t: bits 0-1 inside a thread, the rest
// through shared memory (one barrier per application of H, double buffered).
//
//   k_pauli_prep   per (problem, n): the coefficients of every step, cx_b = sum_c u_c ax[c][b] and
//                  cy_b (FP64, stored in the propagation precision), their bound sum_b |cx_b| + |cy_b|
//                  on the sub-interval, and the Chebyshev parameters.
//   k_pauli_sweep  Algorithm 1 (a)-(b): psi forward and chi backward (two CTAs per problem), the
//                  FP64 states at the partition.
//   k_pauli_sub    Algorithm 1 (c): per (problem, n) the sub-problem state forward (stored per
//                  step), the adjoint backward and, per step, the 2q overlaps <chi|X_b psi>,
//                  <chi|Y_b psi>; then the gradient of every control (trapezoid rule of Eq. (gradJ)),
//                  Err and the ascent step of Eq. (gradStep).
#include "ism_large.cuh"
#include "ism_launch.h"

namespace ism {

constexpr int PQMAX = 10;   // bits (d <= 1024)
constexpr int PMMAX = 32;   // controls

// Exchange of a CTA-wide state through shared memory (the layout of OpBitflipCTA's 4-element path):
// element pairs (0,1) of every thread in [0, D/2), pairs (2,3) in [D/2, D).
template <typename R, int D, class V>
__device__ __forceinline__ void xstore(typename C2<R>::T* b, const V& in) {
  const int t = threadIdx.x;
  if constexpr (sizeof(R) == 4) {
    float4* b4 = reinterpret_cast<float4*>(b);
    b4[t] = make_float4(in.re[0], in.im[0], in.re[1], in.im[1]);
    b4[D / 4 + t] = make_float4(in.re[2], in.im[2], in.re[3], in.im[3]);
  } else {
    typename C2<R>::T z0, z1, z2, z3;
    z0.x = in.re[0]; z0.y = in.im[0]; z1.x = in.re[1]; z1.y = in.im[1];
    z2.x = in.re[2]; z2.y = in.im[2]; z3.x = in.re[3]; z3.y = in.im[3];
    b[2 * t] = z0; b[2 * t + 1] = z1;
    b[D / 2 + 2 * t] = z2; b[D / 2 + 2 * t + 1] = z3;
  }
}
template <typename R, int D>
__device__ __forceinline__ void xload(const typename C2<R>::T* b, int tp, typename C2<R>::T (&p)[4]) {
  if constexpr (sizeof(R) == 4) {
    const float4* b4 = reinterpret_cast<const float4*>(b);
    const float4 lo4 = b4[tp], hi4 = b4[D / 4 + tp];
    p[0].x = lo4.x; p[0].y = lo4.y; p[1].x = lo4.z; p[1].y = lo4.w;
    p[2].x = hi4.x; p[2].y = hi4.y; p[3].x = hi4.z; p[3].y = hi4.w;
  } else {
    p[0] = b[2 * tp]; p[1] = b[2 * tp + 1]; p[2] = b[D / 2 + 2 * tp]; p[3] = b[D / 2 + 2 * tp + 1];
  }
}

template <typename R, int W_>
struct OpPauliCTA {
  static constexpr int W = W_, E = 4, NT = 32 * W_;
  static constexpr int LW = Log2<W_>::v, Q = 7 + LW, D = 1 << Q;
  using R2 = typename C2<R>::T;
  R ah[4], al[4];   // 2(H0_ee - c)/rad as hi + lo
  R yx[Q], yy[Q];   // 2 cx_b / rad, 2 cy_b / rad of the current step
  R2* buf;          // [2][D] exchange buffers in shared memory
  mutable int par;

  __device__ void load(R2* sbuf) {
    buf = sbuf;
    par = 0;
  }
  // The next exchange buffer, for an exchange of the caller's own between two applications of H
  // (the double-buffering argument of flips then covers it too).
  __device__ __forceinline__ R2* next_buf() const {
    R2* b = buf + par * D;
    par ^= 1;
    return b;
  }
  __device__ void scale(const double* H0d, const Cheb<R>& ch) {
#pragma unroll
    for (int r = 0; r < 4; ++r) split2<R>((H0d[threadIdx.x * 4 + r] - ch.cd) * ch.s2d, ah[r], al[r]);
  }
  // row: the step's coefficients [cx_0 .. cx_{Q-1}, cy_0 .. cy_{Q-1}]
  __device__ __forceinline__ void set_step(const R* row, const Cheb<R>& ch) {
    const R s2 = R(2) * ch.inv_rad;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      yx[i] = __ldg(row + i) * s2;
      yy[i] = __ldg(row + Q + i) * s2;
    }
  }
  // acc += sum_b (wx_b X_b + wy_b Y_b) in.  Every thread of the CTA calls this in the same order.
  template <class V>
  __device__ __forceinline__ void flips(const V& in, V& acc, const R* wx, const R* wy) const {
    const int t = threadIdx.x;
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const R sy = ((r >> i) & 1) ? wy[i] : -wy[i];
        const R pr = in.re[r ^ (1 << i)], pi = in.im[r ^ (1 << i)];
        acc.re[r] = fma(wx[i], pr, fma(-sy, pi, acc.re[r]));
        acc.im[r] = fma(wx[i], pi, fma(sy, pr, acc.im[r]));
      }
    R2* b = next_buf();
    xstore<R, D>(b, in);
    __syncthreads();
#pragma unroll
    for (int i = 2; i < Q; ++i) {
      R2 p[4];
      xload<R, D>(b, t ^ (1 << (i - 2)), p);
      const R sy = ((t >> (i - 2)) & 1) ? wy[i] : -wy[i];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        acc.re[r] = fma(wx[i], p[r].x, fma(-sy, p[r].y, acc.re[r]));
        acc.im[r] = fma(wx[i], p[r].y, fma(sy, p[r].x, acc.im[r]));
      }
    }
  }
  template <class V>
  __device__ __forceinline__ void rec(const V& in, const V& sub, V& out) const {
    V t;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      R xr = -sub.re[r], xi = -sub.im[r];
      if (sizeof(R) == 4) { xr = fma(al[r], in.re[r], xr); xi = fma(al[r], in.im[r], xi); }
      t.re[r] = fma(ah[r], in.re[r], xr);
      t.im[r] = fma(ah[r], in.im[r], xi);
    }
    flips(in, t, yx, yy);
    out = t;
  }
};

// ----------------------------------------------------------------------------- k_pauli_prep
template <typename R>
__global__ void __launch_bounds__(32) k_pauli_prep(KParams p) {
  const int n = blockIdx.x, b = blockIdx.y, lane = threadIdx.x;
  const int j0 = p.jn[n], j1 = p.jn[n + 1], m = p.m, q = p.q;
  __shared__ double wts[PMMAX * PQMAX * 2];
  for (int i = lane; i < m * q * 2; i += 32) wts[i] = p.wts[i];
  __syncwarp();
  const double* ub = p.u + (long)b * p.Nt * m;
  R* cb = reinterpret_cast<R*>(p.cxy) + (long)b * p.Nt * 2 * q;
  double um = 0.0;
  for (int j = j0 + lane; j < j1; j += 32) {
    double cx[PQMAX], cy[PQMAX];
    for (int i = 0; i < q; ++i) { cx[i] = 0.0; cy[i] = 0.0; }
    for (int c = 0; c < m; ++c) {
      const double uc = ub[(long)j * m + c];
      if (!isfinite(uc)) atomicOr(p.status, ST_NONFINITE);
      for (int i = 0; i < q; ++i) {
        cx[i] = fma(uc, wts[(c * q + i) * 2], cx[i]);
        cy[i] = fma(uc, wts[(c * q + i) * 2 + 1], cy[i]);
      }
    }
    double s = 0.0;
    for (int i = 0; i < q; ++i) {
      s += fabs(cx[i]) + fabs(cy[i]);
      cb[(long)j * 2 * q + i] = (R)cx[i];
      cb[(long)j * 2 * q + q + i] = (R)cy[i];
    }
    um = s > um ? s : um;
  }
  for (int o = 16; o >= 1; o >>= 1) {
    const double x = __shfl_xor_sync(0xffffffffu, um, o);
    um = x > um ? x : um;
  }
  __shared__ Cheb<R> ch;
  cheb_params<R>(ch, p.ctab, p.tau, p.c0, p.r0, 1.0, um, p.tol, p.phase[n], p.status);
  __syncwarp();
  const int* src = reinterpret_cast<const int*>(&ch);
  int* dst = reinterpret_cast<int*>(const_cast<void*>(p.cheb)) + ((long)b * p.N + n) * (sizeof(Cheb<R>) / sizeof(int));
  for (int i = lane; i < (int)(sizeof(Cheb<R>) / sizeof(int)); i += 32) dst[i] = src[i];
}

// ---------------------------------------------------------------------------- k_pauli_sweep
// grid (2, B): CTA 0 propagates psi forward from psi_i, CTA 1 chi backward from psi_f (overlap
// objective), both compensated in FP32 and rounded through FP64 at every sub-interval end.
template <typename R, int W>
__global__ void __launch_bounds__(32 * W) k_pauli_sweep(KParams p) {
  using Op = OpPauliCTA<R, W>;
  constexpr int E = 4, D = Op::D, Q = Op::Q;
  constexpr bool COMP = sizeof(R) == 4;
  using R2 = typename C2<R>::T;
  __shared__ __align__(16) R2 sbuf[2 * D];
  __shared__ Cheb<R> ch;
  const int b = blockIdx.y, N = p.N;
  const R* cb = reinterpret_cast<const R*>(p.cxy) + (long)b * p.Nt * 2 * Q;
  double2* psin = p.psin_w + (long)b * (N + 1) * D;
  double2* chin = p.chin_w + (long)b * (N + 1) * D;
  Op op;
  op.load(sbuf);
  Vec<R, E> v, lo;
  if (blockIdx.x == 0) {
    load_state<R, E>(v, lo, p.psi_i);
#pragma unroll
    for (int r = 0; r < E; ++r) psin[threadIdx.x * E + r] = p.psi_i[threadIdx.x * E + r];
    for (int n = 0; n < N; ++n) {
      cheb_load_cta<R>(ch, p.cheb, (long)b * N + n);
      op.scale(p.H0d, ch);
      const int j0 = p.jn[n], j1 = p.jn[n + 1];
      for (int j = j0; j < j1; ++j) {
        op.set_step(cb + (long)j * 2 * Q, ch);
        cheb_step<false, COMP>(v, lo, op, ch, ch.K, ch.S);
      }
      phase_store<R, E>(v, lo, ch, false, psin + (long)(n + 1) * D);
      if (p.count && threadIdx.x == 0) count_work<R>(p.count, ch, j1 - j0, 0);
    }
  } else {
    double2* chT = chin + (long)N * D;
#pragma unroll
    for (int r = 0; r < E; ++r) chT[threadIdx.x * E + r] = p.psi_f[threadIdx.x * E + r];
    load_state<R, E>(v, lo, p.psi_f);
    for (int n = N - 1; n >= 0; --n) {
      cheb_load_cta<R>(ch, p.cheb, (long)b * N + n);
      op.scale(p.H0d, ch);
      const int j0 = p.jn[n], j1 = p.jn[n + 1];
      for (int j = j1 - 1; j >= j0; --j) {
        op.set_step(cb + (long)j * 2 * Q, ch);
        cheb_step<true, COMP>(v, lo, op, ch, ch.K, ch.S);
      }
      phase_store<R, E>(v, lo, ch, true, chin + (long)n * D);
      if (p.count && threadIdx.x == 0) count_work<R>(p.count, ch, j1 - j0, 0);
    }
  }
}

// ------------------------------------------------------------------------------ k_pauli_sub
// grid (N, B): sub-problem n of problem b, the two forms of k_subfwd / k_subinterval.  Slot s of the
// sub-interval (s = 0..ns) receives the 2q overlaps <a_s|X_b psi_s>, <a_s|Y_b psi_s> in zq, a = chi
// (form 1: psi and chi carried forward from psi(t_n), chi(t_n), nothing per step stored) or a = delta
// (form 0: the literal sub-problem's adjoint in the delta form; psi_n checkpointed every p.cks steps
// and each segment's states recomputed from its checkpoint into a buffer of p.cks states).
template <typename R, int W>
__global__ void __launch_bounds__(32 * W) k_pauli_sub(KParams p) {
  using Op = OpPauliCTA<R, W>;
  constexpr int E = 4, D = Op::D, Q = Op::Q, NT = 32 * W;
  constexpr bool COMP = sizeof(R) == 4;
  constexpr int CKP = COMP ? 2 : 1;
  using R2 = typename C2<R>::T;
  __shared__ __align__(16) R2 sbuf[2 * D];
  __shared__ R2 zred[W][2 * Q];
  __shared__ double wsm[PMMAX * PQMAX * 2];
  __shared__ Cheb<R> ch;
  __shared__ double red[32];
  const int n = blockIdx.x, b = blockIdx.y, t = threadIdx.x, lane = t & 31, wid = t >> 5;
  const int j0 = p.jn[n], j1 = p.jn[n + 1], ns = j1 - j0, m = p.m;
  const long gid = (long)b * p.N + n;
  const double beta = p.beta[n];
  for (int i = t; i < m * Q * 2; i += NT) wsm[i] = p.wts[i];
  cheb_load_cta<R>(ch, p.cheb, gid);
  const R* cb = reinterpret_cast<const R*>(p.cxy) + (long)b * p.Nt * 2 * Q;
  Op op;
  op.load(sbuf);
  op.scale(p.H0d, ch);
  const int K = ch.K, S = ch.S;
  const long off_n = ((long)b * (p.N + 1) + n) * D;
  const long slot0 = (long)b * (p.Nt + p.N) + j0 + n;
  R2* zq0 = reinterpret_cast<R2*>(p.zq) + slot0 * 2 * Q;         // slot s at zq0 + s*2Q

  // ---- overlaps <a|X_b ps>, <a|Y_b ps> for every bit b into slot s (FP32 products in mixed mode):
  // ps goes through the op's next exchange buffer; each bit's four partial sums are reduced over the
  // warp at once, the W warp partials summed by 2Q threads after one barrier.
  auto overlaps = [&](int s, const Vec<R, E>& a, const Vec<R, E>& ps) {
    R2* xb = op.next_buf();
    xstore<R, D>(xb, ps);
    __syncthreads();
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      R2 pp[4];
      if (i < 2) {
#pragma unroll
        for (int r = 0; r < 4; ++r) { pp[r].x = ps.re[r ^ (1 << i)]; pp[r].y = ps.im[r ^ (1 << i)]; }
      } else {
        xload<R, D>(xb, t ^ (1 << (i - 2)), pp);
      }
      R ax = R(0), bx = R(0), ay = R(0), by = R(0);
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        // conj(a) p = A + i B;  conj(a) (i s p) = -s B + i s A
        const R A = fma(a.re[r], pp[r].x, a.im[r] * pp[r].y);
        const R Bv = fma(a.re[r], pp[r].y, -a.im[r] * pp[r].x);
        const bool set = i < 2 ? ((r >> i) & 1) : ((t >> (i - 2)) & 1);
        ax += A;
        bx += Bv;
        ay += set ? -Bv : Bv;
        by += set ? A : -A;
      }
#pragma unroll
      for (int o = 16; o >= 1; o >>= 1) {
        ax += __shfl_xor_sync(0xffffffffu, ax, o);
        bx += __shfl_xor_sync(0xffffffffu, bx, o);
        ay += __shfl_xor_sync(0xffffffffu, ay, o);
        by += __shfl_xor_sync(0xffffffffu, by, o);
      }
      if (lane == 0) {
        R2 x, y;
        x.x = ax; x.y = bx;
        y.x = ay; y.y = by;
        zred[wid][i] = x;
        zred[wid][Q + i] = y;
      }
    }
    __syncthreads();
    if (t < 2 * Q) {
      R sr = R(0), si = R(0);
#pragma unroll
      for (int w = 0; w < W; ++w) { sr += zred[w][t].x; si += zred[w][t].y; }
      R2 z; z.x = sr; z.y = si;
      zq0[(long)s * 2 * Q + t] = z;
    }
  };

  double nrm = 0.0, cPhi = 1.0, sPhi = 0.0;
  if (p.form) {
    Vec<R, E> a, alo, c, clo;
    load_state<R, E>(a, alo, p.psin + off_n);
    load_state<R, E>(c, clo, p.chin + off_n);
    for (int s = 0; s < ns; ++s) {
      overlaps(s, c, a);
      op.set_step(cb + (long)(j0 + s) * 2 * Q, ch);
      cheb_step<false, COMP>(a, alo, op, ch, K, S);
      cheb_step<false, COMP>(c, clo, op, ch, K, S);
    }
    overlaps(ns, c, a);
    // |delta(t_{n+1})|^2, delta = (chi - psi)(t_{n+1}) / beta_n from the FP64 boundary states
#pragma unroll
    for (int r = 0; r < E; ++r) {
      const int e = t * E + r;
      const double2 x = p.chin[off_n + D + e], y = p.psin[off_n + D + e];
      const double dr = (x.x - y.x) / beta, di = (x.y - y.y) / beta;
      nrm += dr * dr + di * di;
    }
    nrm = cta_sum(nrm, red);
  } else {
    sPhi = ch.sph;
    cPhi = ch.cph;
    const int SC = p.cks;
    R2* ck = reinterpret_cast<R2*>(p.ckpt) + gid * (long)p.nck * CKP * D + t * E;
    R2* sb = reinterpret_cast<R2*>(p.segb) + gid * (long)SC * D + t * E;
    const double2* phn1 = p.phi + off_n + D;
    Vec<R, E> v, lo;
    load_state<R, E>(v, lo, p.phi + off_n);
    // ---- forward sweep: checkpoints
    for (int s = 0; s < ns; ++s) {
      if (s % SC == 0) {
        R2* c = ck + (long)(s / SC) * CKP * D;
#pragma unroll
        for (int r = 0; r < E; ++r) {
          R2 z; z.x = v.re[r]; z.y = v.im[r]; c[r] = z;
          if (COMP) { R2 y; y.x = lo.re[r]; y.y = lo.im[r]; c[D + r] = y; }
        }
      }
      op.set_step(cb + (long)(j0 + s) * 2 * Q, ch);
      cheb_step<false, COMP>(v, lo, op, ch, K, S);
    }
    // ---- terminal residual delta = phi_{n+1} - psi_n(t_{n+1}) in FP64
    Vec<R, E> dl;
#pragma unroll
    for (int r = 0; r < E; ++r) {
      const int e = t * E + r;
      const double2 z = phn1[e];
      double pr, pi;
      phase_rotate(cPhi, sPhi, false, (double)v.re[r] + (double)lo.re[r], (double)v.im[r] + (double)lo.im[r], pr, pi);
      const double dr = z.x - pr, di = z.y - pi;
      dl.re[r] = (R)dr;
      dl.im[r] = (R)di;
      nrm += dr * dr + di * di;
    }
    nrm = cta_sum(nrm, red);
    overlaps(ns, dl, v);
    // ---- backward sweep over the segments, last to first
    const int nck = (ns + SC - 1) / SC;
    for (int c = nck - 1; c >= 0; --c) {
      const int s0 = c * SC, s1 = min(s0 + SC, ns);
      {
        Vec<R, E> x, xl;
        const R2* cc = ck + (long)c * CKP * D;
#pragma unroll
        for (int r = 0; r < E; ++r) {
          const R2 z = cc[r];
          x.re[r] = z.x; x.im[r] = z.y;
          if (COMP) { const R2 y = cc[D + r]; xl.re[r] = y.x; xl.im[r] = y.y; }
          else { xl.re[r] = R(0); xl.im[r] = R(0); }
        }
        for (int s = s0; s < s1; ++s) {
#pragma unroll
          for (int r = 0; r < E; ++r) { R2 z; z.x = x.re[r]; z.y = x.im[r]; sb[(long)(s - s0) * D + r] = z; }
          if (s + 1 < s1) {
            op.set_step(cb + (long)(j0 + s) * 2 * Q, ch);
            cheb_step<false, COMP>(x, xl, op, ch, K, S);
          }
        }
      }
      for (int s = s1 - 1; s >= s0; --s) {
        op.set_step(cb + (long)(j0 + s) * 2 * Q, ch);
        cheb_step<true>(dl, op, ch, K, S);
        Vec<R, E> ps;
#pragma unroll
        for (int r = 0; r < E; ++r) { const R2 z = sb[(long)(s - s0) * D + r]; ps.re[r] = z.x; ps.im[r] = z.y; }
        overlaps(s, dl, ps);
      }
    }
  }
  __syncthreads();   // every slot's overlaps are written

  // ---- FP64 pass over the steps: every control's gradient (trapezoid), Err, ascent step
  const double ht = 0.5 * p.tau * p.w / ((p.form && !p.global) ? beta : 1.0);
  const double step = p.rho * beta / p.tau;
  double* ub = p.u + (long)b * p.Nt * m;
  double* gb = p.grad + (long)b * p.Nt * m;
  double err = 0.0;
  for (int s = t; s < ns; s += NT) {
    const int j = j0 + s;
    double Ix[Q], Iy[Q];   // Im(exp(-i Phi) z) summed over the two ends of step j
#pragma unroll
    for (int i = 0; i < Q; ++i) {
      const R2 xa = zq0[(long)s * 2 * Q + i], xb = zq0[(long)(s + 1) * 2 * Q + i];
      const R2 ya = zq0[(long)s * 2 * Q + Q + i], yb = zq0[(long)(s + 1) * 2 * Q + Q + i];
      Ix[i] = cPhi * ((double)xa.y + (double)xb.y) - sPhi * ((double)xa.x + (double)xb.x);
      Iy[i] = cPhi * ((double)ya.y + (double)yb.y) - sPhi * ((double)ya.x + (double)yb.x);
    }
    for (int c = 0; c < m; ++c) {
      double acc = 0.0;
#pragma unroll
      for (int i = 0; i < Q; ++i) acc = fma(wsm[(c * Q + i) * 2], Ix[i], fma(wsm[(c * Q + i) * 2 + 1], Iy[i], acc));
      const double g = ht * acc;
      err += fabs(g);
      gb[(long)j * m + c] = g;
      if (p.update) ub[(long)j * m + c] += step * g;
    }
  }
  err = cta_sum(err, red);
  if (t == 0) {
    if (p.Jn) p.Jn[gid] = p.w * (-0.5 * nrm);
    if (p.err) p.err[gid] = err;
    count_work<R>(p.count, ch, p.form ? 2L * ns : 3L * ns - (ns + p.cks - 1) / p.cks, 0);
  }
}

template <typename R>
cudaError_t launch_pauli_prep_t(const KParams& p, cudaStream_t st) {
  k_pauli_prep<R><<<dim3(p.N, p.B), 32, 0, st>>>(p);
  return cudaGetLastError();
}
template <typename R, int W>
cudaError_t launch_pauli_sweep_t(const KParams& p, cudaStream_t st) {
  k_pauli_sweep<R, W><<<dim3(2, p.B), 32 * W, 0, st>>>(p);
  return cudaGetLastError();
}
template <typename R, int W>
cudaError_t launch_pauli_sub_t(const KParams& p, cudaStream_t st) {
  k_pauli_sub<R, W><<<dim3(p.N, p.B), 32 * W, 0, st>>>(p);
  return cudaGetLastError();
}

template <typename R, int W>
static void fill_pauli(KernelSet* ks) {
  ks->large = true;
  ks->prep = &launch_pauli_prep_t<R>;
  ks->lsweep = &launch_pauli_sweep_t<R, W>;
  ks->subinterval = &launch_pauli_sub_t<R, W>;
  ks->G = 32 * W;
  ks->E = 4;
  ks->W = W;
}

template <typename R>
static bool pick(int d, KernelSet* ks) {
  switch (d) {
    case 128: fill_pauli<R, 1>(ks); return true;
    case 256: fill_pauli<R, 2>(ks); return true;
    case 512: fill_pauli<R, 4>(ks); return true;
    case 1024: fill_pauli<R, 8>(ks); return true;
    default: return false;
  }
}

bool kernels_pauli(int prec, int d, KernelSet* ks) { return prec == 0 ? pick<double>(d, ks) : pick<float>(d, ks); }

}  // namespace ism
