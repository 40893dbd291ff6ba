// ism_device.cuh -- device building blocks of the ISM propagation kernels (sm_103a).
//
// A state vector of dimension d lives in the registers of a "group" of G consecutive lanes of one
// warp, E contiguous elements per lane (element e = lane_in_group * E + r, r = 0..E-1, zero padded
// up to G*E).  Real and imaginary parts are separate register arrays: every Hamiltonian here is real
// symmetric, so H acts on them independently.
//
// One time step applies U_j = exp(-i tau H(u_j)), H(u) = H0 + u H1 (Sec. 2, Eq. (dir)), by the
// Chebyshev expansion of the exponential (Jacobi-Anger):
//     exp(-i x Y) = sum_k a_k (-i)^k T_k(Y),  a_0 = J_0(x), a_k = 2 J_k(x),
// with Y = (H - c)/rad scaled into [-1, 1] (c, rad from Gershgorin bounds of H0 and H1 and the
// largest |u| of the sub-interval), x = tau * rad, T_{k+1} = 2 Y T_k - T_{k-1}, and the global phase
// exp(-i tau c).  J_k(x) is summed from its power series (Abramowitz & Stegun 9.1.10) in FP64.
// The adjoint step U_j^H uses (+i)^k and exp(+i tau c).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace ism {

constexpr int KMAX = 32;        // Chebyshev terms held per group
constexpr double XMAX = 4.0;    // largest tau*rad per sub-step (more -> sub-steps)

enum StatusBits : int {
  ST_TIMEOUT = 1,      // a bounded mbarrier wait gave up
  ST_KOVERFLOW = 2,    // Chebyshev series needed more than KMAX terms
  ST_NONFINITE = 4,    // NaN/Inf met in a control or a result
};

template <typename R> struct C2;
template <> struct C2<float> { using T = float2; };
template <> struct C2<double> { using T = double2; };

// ------------------------------------------------------------------------- group shuffles
// All calls use the full-warp mask: every lane of the warp executes them (loop trip counts are
// made warp-uniform by the callers).
template <int G, typename T> __device__ __forceinline__ T g_up(T v) { return __shfl_up_sync(0xffffffffu, v, 1, G); }
template <int G, typename T> __device__ __forceinline__ T g_down(T v) { return __shfl_down_sync(0xffffffffu, v, 1, G); }
template <int G, typename T> __device__ __forceinline__ T g_xor(T v, int m) { return __shfl_xor_sync(0xffffffffu, v, m, G); }
template <int G, typename T> __device__ __forceinline__ T g_idx(T v, int s) { return __shfl_sync(0xffffffffu, v, s, G); }

template <int G, typename T> __device__ __forceinline__ T g_sum(T v) {
#pragma unroll
  for (int m = G / 2; m >= 1; m >>= 1) v += g_xor<G>(v, m);
  return v;
}
template <int G, typename T> __device__ __forceinline__ T g_max(T v) {
#pragma unroll
  for (int m = G / 2; m >= 1; m >>= 1) { T o = g_xor<G>(v, m); v = o > v ? o : v; }
  return v;
}
__device__ __forceinline__ int warp_max_i(int v) { return __reduce_max_sync(0xffffffffu, (unsigned)v); }

template <typename R, int E> struct Vec { R re[E]; R im[E]; };

// --------------------------------------------------------------- Bessel and Chebyshev set-up
// J_k(x) from the ascending series sum_m (-1)^m (x/2)^(2m+k) / (m! (m+k)!), 0 <= x <= XMAX.
__device__ inline double bessel_jk(int k, double x) {
  const double h = 0.5 * x;
  double t = 1.0;
  for (int i = 1; i <= k; ++i) t *= h / (double)i;
  double s = t;
  const double h2 = h * h;
  for (int m = 1; m < 60; ++m) {
    t *= -h2 / ((double)m * (double)(m + k));
    s += t;
    if (fabs(t) <= 1e-18 * fabs(s)) break;
  }
  return s;
}

// Per-group propagator parameters (shared memory).  cf[k] carries a_k with the sign of (-i)^k folded
// in: even k -> a_k (-1)^(k/2) multiplies the vector itself, odd k -> a_k (-1)^((k-1)/2) multiplies
// -i times the vector (forward); the adjoint flips the odd terms.
template <typename R> struct Cheb {
  R cf[KMAX];
  R cph, sph;       // cos, sin of tau_s * c
  R c, inv_rad;     // spectral centre and 1/rad
  int K, S;         // terms, sub-steps per time step
};

// Fill `ch` for a group whose controls satisfy |u| <= umax.  All lanes of the warp must call this
// (K and S are made warp-uniform).  lg = lane in group.
template <int G, typename R>
__device__ void cheb_setup(Cheb<R>& ch, int lg, double tau, double c0, double r0, double h1n,
                          double umax, double tol, int* status) {
  double rad = (r0 + umax * h1n) * (1.0 + 1e-12) + 1e-12;
  double x = tau * rad;
  int S = (int)ceil(x / XMAX);
  if (S < 1) S = 1;
  S = warp_max_i(S);
  const double xs = x / (double)S;
  int kneed = 0;
  for (int k = lg; k < KMAX; k += G) {
    double a = bessel_jk(k, xs) * (k == 0 ? 1.0 : 2.0);
    if (fabs(a) >= tol) kneed = k + 1 > kneed ? k + 1 : kneed;
    double sg = ((k >> 1) & 1) ? -1.0 : 1.0;   // (-1)^(k/2) for even k, (-1)^((k-1)/2) for odd k
    ch.cf[k] = (R)(sg * a);
  }
  kneed = g_max<G>(kneed);
  if (kneed >= KMAX && lg == 0) atomicOr(status, ST_KOVERFLOW);
  int K = kneed < 2 ? 2 : kneed;
  K = warp_max_i(K);
  if (lg == 0) {
    double sn, cs;
    sincos(tau / (double)S * c0, &sn, &cs);
    ch.cph = (R)cs;
    ch.sph = (R)sn;
    ch.c = (R)c0;
    ch.inv_rad = (R)(1.0 / rad);
    ch.K = K;
    ch.S = S;
  }
  __syncwarp();
}

// ---------------------------------------------------------------------- Hamiltonian structures
// Each op offers, per lane:
//   set_u(u, ch): prepare Y(u) = (H0 + u H1 - c)/rad for the lane's rows (scaled by 2 for the recurrence)
//   rec(in, sub, out): out = 2 Y in - sub
//   h1(in, out):       out = H1 in
// Packed layouts in global memory (element type R):
//   Tridiag: [d0 (d) | o0 (d) | d1 (d) | o1 (d)], o[e] couples e and e+1, o[d-1] = 0.
//   Bitflip: [d0 (d) | h (q)], H1 = sum_i h_i X_i, d = 2^q = G*E.
//   Dense:   [(G E) x (G E) pairs {H0_ef, H1_ef}] zero padded, row-major, staged in shared memory.

template <typename R, int G_, int E_>
struct OpTridiag {
  static constexpr int G = G_, E = E_, DP_SMEM = 0;
  R d0[E], d1[E], o0[E], o1[E];
  R yd[E], yo[E], yom;   // 2Y diagonal, 2Y off-diagonal (e, e+1), 2Y off-diagonal (e0-1, e0)
  R h1m;                  // H1 off-diagonal (e0-1, e0)

  __device__ void load(const R* H, int d, int lg, void*) {
#pragma unroll
    for (int r = 0; r < E; ++r) {
      int e = lg * E + r;
      bool in = e < d;
      d0[r] = in ? H[e] : R(0);
      o0[r] = in ? H[d + e] : R(0);
      d1[r] = in ? H[2 * d + e] : R(0);
      o1[r] = in ? H[3 * d + e] : R(0);
    }
    R t = g_up<G>(o1[E - 1]);
    h1m = lg == 0 ? R(0) : t;
  }
  __device__ __forceinline__ void set_u(R u, const Cheb<R>& ch, int lg) {
    const R s2 = R(2) * ch.inv_rad;
#pragma unroll
    for (int r = 0; r < E; ++r) {
      yd[r] = (d0[r] + u * d1[r] - ch.c) * s2;
      yo[r] = (o0[r] + u * o1[r]) * s2;
    }
    R t = g_up<G>(yo[E - 1]);
    yom = lg == 0 ? R(0) : t;
  }
  template <class V>
  __device__ __forceinline__ void rec(const V& in, const V& sub, V& out) const {
    R lre = g_up<G>(in.re[E - 1]), lim = g_up<G>(in.im[E - 1]);
    R rre = g_down<G>(in.re[0]), rim = g_down<G>(in.im[0]);
#pragma unroll
    for (int r = 0; r < E; ++r) {
      R mre = r == 0 ? lre : in.re[r - 1], mim = r == 0 ? lim : in.im[r - 1];
      R pre = r == E - 1 ? rre : in.re[r + 1], pim = r == E - 1 ? rim : in.im[r + 1];
      R ym = r == 0 ? yom : yo[r - 1];
      out.re[r] = fma(yd[r], in.re[r], fma(ym, mre, fma(yo[r], pre, -sub.re[r])));
      out.im[r] = fma(yd[r], in.im[r], fma(ym, mim, fma(yo[r], pim, -sub.im[r])));
    }
  }
  template <class V>
  __device__ __forceinline__ void h1(const V& in, V& out) const {
    R lre = g_up<G>(in.re[E - 1]), lim = g_up<G>(in.im[E - 1]);
    R rre = g_down<G>(in.re[0]), rim = g_down<G>(in.im[0]);
#pragma unroll
    for (int r = 0; r < E; ++r) {
      R mre = r == 0 ? lre : in.re[r - 1], mim = r == 0 ? lim : in.im[r - 1];
      R pre = r == E - 1 ? rre : in.re[r + 1], pim = r == E - 1 ? rim : in.im[r + 1];
      R om = r == 0 ? h1m : o1[r - 1];
      out.re[r] = fma(d1[r], in.re[r], fma(om, mre, o1[r] * pre));
      out.im[r] = fma(d1[r], in.im[r], fma(om, mim, o1[r] * pim));
    }
  }
};

template <int E> struct Log2 { static constexpr int v = E <= 1 ? 0 : 1 + Log2<E / 2>::v; };
template <> struct Log2<1> { static constexpr int v = 0; };

template <typename R, int G_, int E_>
struct OpBitflip {
  static constexpr int G = G_, E = E_, DP_SMEM = 0;
  static constexpr int LE = Log2<E>::v, LG = Log2<G>::v, Q = LE + LG;
  R d0[E], yd[E];
  R h[Q > 0 ? Q : 1];
  R yh[Q > 0 ? Q : 1];

  __device__ void load(const R* H, int d, int lg, void*) {
#pragma unroll
    for (int r = 0; r < E; ++r) d0[r] = H[lg * E + r];
#pragma unroll
    for (int i = 0; i < Q; ++i) h[i] = H[d + i];
  }
  __device__ __forceinline__ void set_u(R u, const Cheb<R>& ch, int) {
    const R s2 = R(2) * ch.inv_rad;
#pragma unroll
    for (int r = 0; r < E; ++r) yd[r] = (d0[r] - ch.c) * s2;
#pragma unroll
    for (int i = 0; i < Q; ++i) yh[i] = u * h[i] * s2;
  }
  template <class V>
  __device__ __forceinline__ void flips(const V& in, V& acc, const R* w) const {
#pragma unroll
    for (int i = 0; i < LE; ++i) {
#pragma unroll
      for (int r = 0; r < E; ++r) {
        acc.re[r] = fma(w[i], in.re[r ^ (1 << i)], acc.re[r]);
        acc.im[r] = fma(w[i], in.im[r ^ (1 << i)], acc.im[r]);
      }
    }
#pragma unroll
    for (int i = LE; i < Q; ++i) {
#pragma unroll
      for (int r = 0; r < E; ++r) {
        R xr = g_xor<G>(in.re[r], 1 << (i - LE));
        R xi = g_xor<G>(in.im[r], 1 << (i - LE));
        acc.re[r] = fma(w[i], xr, acc.re[r]);
        acc.im[r] = fma(w[i], xi, acc.im[r]);
      }
    }
  }
  template <class V>
  __device__ __forceinline__ void rec(const V& in, const V& sub, V& out) const {
#pragma unroll
    for (int r = 0; r < E; ++r) {
      out.re[r] = fma(yd[r], in.re[r], -sub.re[r]);
      out.im[r] = fma(yd[r], in.im[r], -sub.im[r]);
    }
    flips(in, out, yh);
  }
  template <class V>
  __device__ __forceinline__ void h1(const V& in, V& out) const {
#pragma unroll
    for (int r = 0; r < E; ++r) { out.re[r] = R(0); out.im[r] = R(0); }
    flips(in, out, h);
  }
};

// Dense real-symmetric H0, H1 staged as {H0_ef, H1_ef} pairs in shared memory (row-major, padded to
// DP = G*E).  The state's elements are broadcast with shuffles.
template <typename R, int G_, int E_>
struct OpDense {
  static constexpr int G = G_, E = E_, DP = G_ * E_, DP_SMEM = G_ * E_;
  using R2 = typename C2<R>::T;
  const R2* Hs;   // shared memory
  int lg;
  R s2h, u2, cs2; // 2/rad, 2u/rad, 2c/rad

  __device__ void load(const R*, int, int lg_, void* smem) {
    Hs = reinterpret_cast<const R2*>(smem);
    lg = lg_;
  }
  __device__ __forceinline__ void set_u(R u, const Cheb<R>& ch, int) {
    s2h = R(2) * ch.inv_rad;
    u2 = u * s2h;
    cs2 = ch.c * s2h;
  }
  template <bool REC, class V>
  __device__ __forceinline__ void mv(const V& in, V& out, R s2) const {
    R ar[E], ai[E];
#pragma unroll
    for (int r = 0; r < E; ++r) { ar[r] = R(0); ai[r] = R(0); }
#pragma unroll 4
    for (int src = 0; src < G; ++src) {
#pragma unroll
      for (int s = 0; s < E; ++s) {
        const int f = src * E + s;
        R vr = g_idx<G>(in.re[s], src), vi = g_idx<G>(in.im[s], src);
#pragma unroll
        for (int r = 0; r < E; ++r) {
          R2 p = Hs[(lg * E + r) * DP + f];
          R y = REC ? fma(u2, p.y, s2 * p.x) : p.y;
          ar[r] = fma(y, vr, ar[r]);
          ai[r] = fma(y, vi, ai[r]);
        }
      }
    }
#pragma unroll
    for (int r = 0; r < E; ++r) { out.re[r] = ar[r]; out.im[r] = ai[r]; }
  }
  template <class V>
  __device__ __forceinline__ void rec(const V& in, const V& sub, V& out) const {
    V t;
    mv<true>(in, t, s2h);
#pragma unroll
    for (int r = 0; r < E; ++r) {
      out.re[r] = fma(-cs2, in.re[r], t.re[r]) - sub.re[r];
      out.im[r] = fma(-cs2, in.im[r], t.im[r]) - sub.im[r];
    }
  }
  template <class V>
  __device__ __forceinline__ void h1(const V& in, V& out) const { mv<false>(in, out, R(0)); }
};

// ------------------------------------------------------------------ Chebyshev propagator step
// v <- U v (ADJ = false) or U^H v (ADJ = true) for the op's current u.  Warp-uniform control flow.
template <bool ADJ, typename R, int E, class Op>
__device__ __forceinline__ void cheb_step(Vec<R, E>& v, const Op& op, const Cheb<R>& ch) {
  const int K = ch.K;
  for (int s = 0; s < ch.S; ++s) {
    Vec<R, E> t0 = v, t1, acc;
    Vec<R, E> zero;
#pragma unroll
    for (int r = 0; r < E; ++r) { zero.re[r] = R(0); zero.im[r] = R(0); }
    op.rec(t0, zero, t1);   // t1 = 2 Y t0
#pragma unroll
    for (int r = 0; r < E; ++r) { t1.re[r] *= R(0.5); t1.im[r] *= R(0.5); }
    const R c0 = ch.cf[0], c1 = ch.cf[1];
#pragma unroll
    for (int r = 0; r < E; ++r) {
      // even term k=0 on the vector, odd term k=1 on -i*vector (forward) / +i*vector (adjoint)
      if (!ADJ) {
        acc.re[r] = fma(c1, t1.im[r], c0 * t0.re[r]);
        acc.im[r] = fma(-c1, t1.re[r], c0 * t0.im[r]);
      } else {
        acc.re[r] = fma(-c1, t1.im[r], c0 * t0.re[r]);
        acc.im[r] = fma(c1, t1.re[r], c0 * t0.im[r]);
      }
    }
    for (int k = 2; k < K; k += 2) {
      Vec<R, E> t2;
      op.rec(t1, t0, t2);   // T_k
      const R ce = ch.cf[k];
#pragma unroll
      for (int r = 0; r < E; ++r) {
        acc.re[r] = fma(ce, t2.re[r], acc.re[r]);
        acc.im[r] = fma(ce, t2.im[r], acc.im[r]);
      }
      if (k + 1 < K) {
        op.rec(t2, t1, t0);   // T_{k+1} into t0
        const R co = ch.cf[k + 1];
#pragma unroll
        for (int r = 0; r < E; ++r) {
          if (!ADJ) {
            acc.re[r] = fma(co, t0.im[r], acc.re[r]);
            acc.im[r] = fma(-co, t0.re[r], acc.im[r]);
          } else {
            acc.re[r] = fma(-co, t0.im[r], acc.re[r]);
            acc.im[r] = fma(co, t0.re[r], acc.im[r]);
          }
        }
        // rotate: (t0, t1) <- (T_k, T_{k+1})
#pragma unroll
        for (int r = 0; r < E; ++r) {
          R a = t2.re[r], b = t2.im[r];
          t1.re[r] = t0.re[r]; t1.im[r] = t0.im[r];
          t0.re[r] = a; t0.im[r] = b;
        }
        // now t0 = T_k, t1 = T_{k+1}
      }
    }
    const R cp = ch.cph, sp = ch.sph;
#pragma unroll
    for (int r = 0; r < E; ++r) {
      if (!ADJ) {   // times exp(-i theta)
        v.re[r] = fma(acc.re[r], cp, acc.im[r] * sp);
        v.im[r] = fma(acc.im[r], cp, -acc.re[r] * sp);
      } else {      // times exp(+i theta)
        v.re[r] = fma(acc.re[r], cp, -acc.im[r] * sp);
        v.im[r] = fma(acc.im[r], cp, acc.re[r] * sp);
      }
    }
  }
}

}  // namespace ism
