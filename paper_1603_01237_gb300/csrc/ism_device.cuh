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
// largest |u| of the sub-interval), x = tau * rad, T_{k+1} = 2 Y T_k - T_{k-1}.  J_k(x) is summed from
// its power series (Abramowitz & Stegun 9.1.10) in FP64.  The adjoint step U_j^H uses (+i)^k.
//
// The global phase exp(-i tau c) of every step is NOT applied here: callers apply the accumulated
// phase exp(-i c t) of a whole segment once, in FP64.  In FP32 propagation the rounding of a per-step
// phase, of the large diagonal (H0_ee - c)/rad and of the leading coefficients a_0, a_1 is the same at
// every step, so it would grow linearly with the number of steps; here those quantities are held as
// FP32 (hi, lo) pairs computed in FP64, and only rounding that varies from step to step remains.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace ism {

constexpr int KMAX = 32;        // Chebyshev terms held per group
constexpr double XMAX = 4.0;    // largest tau*rad per sub-step (more -> sub-steps)
constexpr int SMAX = 64;        // sub-steps per time step before a plan reports ST_SPECTRUM
constexpr int CN_KMAX = 64;     // Jacobi iterations per Crank-Nicolson solve (rho < 1/2, tol >= 1e-19)

enum StatusBits : int {
  ST_TIMEOUT = 1,      // a bounded mbarrier wait gave up
  ST_KOVERFLOW = 2,    // Chebyshev series needed more than KMAX terms
  ST_NONFINITE = 4,    // NaN/Inf met in a control or a result
  ST_SPECTRUM = 8,     // tau * spectral radius beyond SMAX sub-steps (controls too large)
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

// Packed FP32 complex state: (re, im) of an element in one 64-bit register pair.  Every Hamiltonian
// here is real, so both halves of an element meet the same real coefficient and one packed FMA
// (fma.rn.f32x2, sm_100 and later) updates both: half the instructions of the split layout at the
// same FP32 rate.
template <int E> struct VecP { float2 z[E]; };
__device__ __forceinline__ float2 bc2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }

// --------------------------------------------------------------- Bessel and Chebyshev set-up

// Per-group propagator parameters (shared memory).  cf[k] carries a_k with the sign of (-i)^k folded
// in: even k -> a_k (-1)^(k/2) multiplies the vector itself, odd k -> a_k (-1)^((k-1)/2) multiplies
// -i times the vector (forward); the adjoint flips the odd terms.
template <typename R> struct Cheb {
  R cf[KMAX];       // signed a_k (used for k >= 2), high part
  R cl[KMAX];       // low part (FP32 only: the rounding of a_k would repeat at every step)
  R a0h, a0l;       // a_0 as hi + lo
  R c0h, c0l;       // a_0 - 1 as hi + lo (compensated step)
  R a1h, a1l;       // signed a_1 as hi + lo
  R c, inv_rad;     // spectral centre and 1/rad (FP32 copies)
  double cd, s2d;   // spectral centre and 2/rad in FP64
  double cph, sph;  // cos, sin of the sub-interval's global phase c * tau * (number of steps)
  int K, S;         // terms, sub-steps per time step (Crank-Nicolson: Jacobi iterations, 1)
  R h;              // Crank-Nicolson only: tau / 2
  double hd;        // Crank-Nicolson only: tau / 2 in FP64 (hi/lo diagonal coefficients of FP32 steps)
};

template <typename R> __device__ __forceinline__ void split2(double v, R& hi, R& lo) {
  hi = (R)v;
  lo = sizeof(R) == 4 ? (R)(v - (double)hi) : R(0);
}

// Chebyshev parameters of one sub-interval, computed by one warp (lane k evaluates J_k).
// J_k(x) = (x/2)^k sum_m (-x^2/4)^m / (m! (m+k)!) by Horner's rule on the table
// ctab[k * (BESSEL_M + 1) + m] = 1 / (m! (m+k)!) (FP64, built on the host): no divisions on the device,
// whose FP64 rate is low.  umax bounds |u| on the sub-interval; phase = (cos, sin) of the segment's
// global phase c0 tau (steps), computed on the host.
constexpr int BESSEL_M = 24;

template <typename R>
__device__ void cheb_params(Cheb<R>& ch, const double* ctab, double tau, double c0, double r0, double h1n,
                            double umax, double tol, double2 phase, int* status) {
  const int lane = threadIdx.x & 31;
  const double rad = (r0 + umax * h1n) * (1.0 + 1e-6) + 1e-12;
  const double x = tau * rad;
  int S = x < XMAX * SMAX ? (int)ceil(x / XMAX) : SMAX + 1;
  if (S < 1) S = 1;
  if (S > SMAX) {   // |u| beyond what the sub-step budget covers: flag it and keep the work bounded
    if (lane == 0) atomicOr(status, ST_SPECTRUM);
    S = SMAX;
  }
  const double xs = x / (double)S;
  const double y = -0.25 * xs * xs, h = 0.5 * xs;
  // terms of the series needed: |y|^m / (m!)^2 (the k = 0 ratio, the slowest) below 1e-19; FP64
  // work is scarce on this GPU, and small steps need only a few terms (x = 0.13: 6 of 24)
  int M = 1;
  {
    const float ay = (float)fabs(y);
    float t = 1.f;
    while (M < BESSEL_M) {
      t *= ay / (float)(M * M);
      if (t < 1e-19f) break;
      ++M;
    }
  }
  const int k = lane;   // KMAX == 32 == warp size
  const double* c = ctab + k * (BESSEL_M + 1);
  double acc = c[M];
  for (int m = M - 1; m >= 0; --m) acc = fma(acc, y, c[m]);
  double pw = 1.0, base = h;   // h^k by squaring
  for (int e = k; e; e >>= 1) {
    if (e & 1) pw *= base;
    base *= base;
  }
  const double a = acc * pw * (k == 0 ? 1.0 : 2.0);
  int kneed = fabs(a) >= tol ? k + 1 : 0;
  kneed = warp_max_i(kneed);
  if (kneed >= KMAX && lane == 0) atomicOr(status, ST_KOVERFLOW);
  const double sg = ((k >> 1) & 1) ? -1.0 : 1.0;   // (-1)^(k/2) for even k, (-1)^((k-1)/2) for odd k
  // terms beyond the sub-interval's own count carry exactly zero: a group whose warp runs more terms
  // (the largest count of the warp's groups) adds nothing, so a state's rounding does not depend on
  // the states beside it
  split2<R>(k < (kneed < 2 ? 2 : kneed) ? sg * a : 0.0, ch.cf[k], ch.cl[k]);
  if (lane == 0) {
    // a_0 - 1 = sum_{m>=1} y^m / (m!)^2 without cancellation
    double t = ctab[M];
    for (int m = M - 1; m >= 1; --m) t = fma(t, y, ctab[m]);
    const double j0m1 = t * y;
    split2<R>(1.0 + j0m1, ch.a0h, ch.a0l);
    split2<R>(j0m1, ch.c0h, ch.c0l);
    ch.c = (R)c0;
    ch.inv_rad = (R)(1.0 / rad);
    ch.cd = c0;
    ch.s2d = 2.0 / rad;
    ch.cph = phase.x;   // cos, sin of c0 * tau * (steps of the sub-interval), from the host
    ch.sph = phase.y;
    ch.K = kneed < 2 ? 2 : kneed;
    ch.S = S;
  }
  if (lane == 1) split2<R>(a, ch.a1h, ch.a1l);   // a_1 = 2 J_1 (lane 1 holds it)
}

// cheb_params computed by one thread instead of a warp: the same operations for every term k, in the
// same order, so the same bits.  Terms are evaluated from k = 0 until the bound |J_k(x)| <= (x/2)^k / k!
// puts this and every later a_k below tol / 2 (the bound decreases once k > x/2): those carry zero
// anyway, so a sub-interval costs its own series length in FP64 work, not KMAX terms.  sa: KMAX
// doubles of scratch (shared memory).
template <typename R>
__device__ void cheb_params_1(Cheb<R>& ch, double* sa, const double* ctab, double tau, double c0, double r0,
                              double h1n, double umax, double tol, double2 phase, int* status) {
  const double rad = (r0 + umax * h1n) * (1.0 + 1e-6) + 1e-12;
  const double x = tau * rad;
  int S = x < XMAX * SMAX ? (int)ceil(x / XMAX) : SMAX + 1;
  if (S < 1) S = 1;
  if (S > SMAX) {
    atomicOr(status, ST_SPECTRUM);
    S = SMAX;
  }
  const double xs = x / (double)S;
  const double y = -0.25 * xs * xs, h = 0.5 * xs;
  int M = 1;
  {
    const float ay = (float)fabs(y);
    float t = 1.f;
    while (M < BESSEL_M) {
      t *= ay / (float)(M * M);
      if (t < 1e-19f) break;
      ++M;
    }
  }
  int kneed = 0;
  for (int k = 0; k < KMAX; ++k) {
    const double* c = ctab + k * (BESSEL_M + 1);
    double acc = c[M];
    for (int m = M - 1; m >= 0; --m) acc = fma(acc, y, c[m]);
    double pw = 1.0, base = h;   // h^k by squaring
    for (int e = k; e; e >>= 1) {
      if (e & 1) pw *= base;
      base *= base;
    }
    const double a = acc * pw * (k == 0 ? 1.0 : 2.0);
    sa[k] = a;
    if (fabs(a) >= tol) kneed = k + 1;
    if (k >= 1 && (double)k > h && 2.0 * pw * c[0] < 0.5 * tol) break;   // c[0] = 1/k!
  }
  if (kneed >= KMAX) atomicOr(status, ST_KOVERFLOW);
  const int K2 = kneed < 2 ? 2 : kneed;
  for (int k = 0; k < KMAX; ++k) {
    const double sg = ((k >> 1) & 1) ? -1.0 : 1.0;
    split2<R>(k < K2 ? sg * sa[k] : 0.0, ch.cf[k], ch.cl[k]);
  }
  double t = ctab[M];
  for (int m = M - 1; m >= 1; --m) t = fma(t, y, ctab[m]);
  const double j0m1 = t * y;
  split2<R>(1.0 + j0m1, ch.a0h, ch.a0l);
  split2<R>(j0m1, ch.c0h, ch.c0l);
  split2<R>(sa[1], ch.a1h, ch.a1l);
  ch.c = (R)c0;
  ch.inv_rad = (R)(1.0 / rad);
  ch.cd = c0;
  ch.s2d = 2.0 / rad;
  ch.cph = phase.x;
  ch.sph = phase.y;
  ch.K = K2;
  ch.S = S;
}

// Crank-Nicolson parameters of one sub-interval (one thread): K Jacobi iterations per linear solve,
// with rho = (tau/2)(off0 + umax off1) (off0, off1: largest off-diagonal absolute row sums of H0 and
// H1) the contraction of each iteration, so that rho^K <= tol (at most CN_KMAX).  rho >= 1/2 is flagged
// ST_SPECTRUM.
template <typename R>
__device__ void cn_params(Cheb<R>& ch, double tau, double off0, double off1, double umax, double tol, int* status) {
  for (int k = 0; k < KMAX; ++k) { ch.cf[k] = R(0); ch.cl[k] = R(0); }
  ch.a0h = ch.a0l = ch.c0h = ch.c0l = ch.a1h = ch.a1l = R(0);
  ch.c = R(0);
  ch.inv_rad = R(0);
  ch.cd = 0.0;
  ch.s2d = 0.0;
  ch.cph = 1.0;   // no global phase is split off
  ch.sph = 0.0;
  ch.S = 1;
  ch.h = (R)(0.5 * tau);
  ch.hd = 0.5 * tau;
  const double rho = 0.5 * tau * (off0 + umax * off1) * (1.0 + 1e-6);
  int K = 1;
  if (rho >= 0.5) {   // flagged; one iteration keeps the (discarded) results bounded
    atomicOr(status, ST_SPECTRUM);
  } else if (rho > 0.0) {
    K = (int)ceil(log(tol) / log(rho));
    K = K < 1 ? 1 : (K > CN_KMAX ? CN_KMAX : K);
  }
  ch.K = K;
}

// Copy a sub-interval's parameters from global memory into a group's shared copy; K and S are made
// warp-uniform (a group runs extra terms with its own tiny coefficients, and extra sub-steps are
// discarded by the caller's select).  Every lane of the warp calls this.
template <int G, typename R>
__device__ void cheb_load(Cheb<R>& ch, const Cheb<R>* src, int lg, int& Kw, int& Sw) {
  const int* s = reinterpret_cast<const int*>(src);
  int* d = reinterpret_cast<int*>(&ch);
  constexpr int words = sizeof(Cheb<R>) / sizeof(int);
  for (int i = lg; i < words; i += G) d[i] = s[i];
  __syncwarp();
  Kw = warp_max_i(ch.K);
  Sw = warp_max_i(ch.S);
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

// HB: H1 has a non-zero diagonal (otherwise its diagonal is neither stored nor applied).  The
// off-diagonals o0 (H0) and o1 (H1) are read from global memory (L1-resident) once per step, not held
// in registers, to keep the register count of the many-lane assembly low.
template <typename R, int G_, int E_, bool HB = true>
struct OpTridiag {
  static constexpr int G = G_, E = E_, DP_SMEM = 0, SMEM_WORDS = 0;
  static constexpr bool PACKED = true;   // offers rec_p / h1_p on packed FP32 states
  static constexpr bool CN = false;      // time step: Chebyshev series (OpTridiagCN: Crank-Nicolson)
  // resident assembly CTAs per SM to aim for (caps registers at 128 where that costs no spills)
  static constexpr int ASM_MINB = (E_ <= 6 && !HB) ? 4 : 1;
  static constexpr int EB = HB ? E_ : 1;
  const R* o0p;           // H0 off-diagonal of this lane's rows
  const R* o1p;           // H1 off-diagonal of this lane's rows
  R o1[E];                // H1 off-diagonal (h1 applications)
  R d1[EB];               // H1 diagonal
  R ah[E], al[E];         // 2(H0_ee - c)/rad as hi + lo (FP64 set-up)
  R yb[EB], yo[E], yom;   // 2u H1_ee/rad, 2Y off-diagonal (e, e+1), 2Y off-diagonal (e0-1, e0)
  R h1m;                  // H1 off-diagonal (e0-1, e0)
  int dd, e0;
  // packed (c, c) copies of the recurrence coefficients for rec_p (R = float), formed once per step
  float2 ah2[E], al2[E], yo2[E], yb2[EB], yom2;

  // H: packed op data in R; H0d: FP64 diagonal of H0
  __device__ void load(const R* H, const double* H0d, int d, int lg, void*) {
    dd = d;
    e0 = lg * E;
    o0p = H + d;
    o1p = H + 3 * d;
#pragma unroll
    for (int r = 0; r < E; ++r) {
      int e = e0 + r;
      bool in = e < d;
      o1[r] = in ? H[3 * d + e] : R(0);
      if (HB) d1[r] = in ? H[2 * d + e] : R(0);
    }
    R t = g_up<G>(o1[E - 1]);
    h1m = lg == 0 ? R(0) : t;
  }
  __device__ void scale(const double* H0d, int d, int lg, const Cheb<R>& ch) {
#pragma unroll
    for (int r = 0; r < E; ++r) {
      int e = lg * E + r;
      split2<R>(e < d ? (H0d[e] - ch.cd) * ch.s2d : 0.0, ah[r], al[r]);
      if constexpr (sizeof(R) == 4) {
        ah2[r] = bc2((float)ah[r]);
        al2[r] = bc2((float)al[r]);
      }
    }
  }
  __device__ __forceinline__ void set_u(R u, const Cheb<R>& ch, int lg) {
    const R s2 = R(2) * ch.inv_rad;
#pragma unroll
    for (int r = 0; r < E; ++r) {
      const int e = e0 + r;
      const R a = e < dd ? __ldg(o0p + e) : R(0);
      const R b = e < dd ? __ldg(o1p + e) : R(0);
      if (HB) yb[r] = u * d1[r] * s2;
      yo[r] = (a + u * b) * s2;
    }
    R t = g_up<G>(yo[E - 1]);
    yom = lg == 0 ? R(0) : t;
    if constexpr (sizeof(R) == 4) {
#pragma unroll
      for (int r = 0; r < E; ++r) {
        yo2[r] = bc2((float)yo[r]);
        if (HB) yb2[r] = bc2((float)yb[r]);
      }
      yom2 = bc2((float)yom);
    }
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
      R xr = fma(ym, mre, fma(yo[r], pre, -sub.re[r]));
      R xi = fma(ym, mim, fma(yo[r], pim, -sub.im[r]));
      if (sizeof(R) == 4) { xr = fma(al[r], in.re[r], xr); xi = fma(al[r], in.im[r], xi); }
      if (HB) { xr = fma(yb[r], in.re[r], xr); xi = fma(yb[r], in.im[r], xi); }
      out.re[r] = fma(ah[r], in.re[r], xr);
      out.im[r] = fma(ah[r], in.im[r], xi);
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
      R xr = fma(om, mre, o1[r] * pre), xi = fma(om, mim, o1[r] * pim);
      if (HB) { xr = fma(d1[r], in.re[r], xr); xi = fma(d1[r], in.im[r], xi); }
      out.re[r] = xr;
      out.im[r] = xi;
    }
  }
  // packed FP32 forms of rec and h1 (R = float).  DL = false leaves out the low part of the diagonal
  // (for sweeps over one sub-interval, where its rounding does not accumulate).
  template <bool DL = true>
  __device__ __forceinline__ void rec_p(const VecP<E>& in, const VecP<E>& sub, VecP<E>& out) const {
    float2 l, q;
    l.x = g_up<G>(in.z[E - 1].x);
    l.y = g_up<G>(in.z[E - 1].y);
    q.x = g_down<G>(in.z[0].x);
    q.y = g_down<G>(in.z[0].y);
#pragma unroll
    for (int r = 0; r < E; ++r) {
      const float2 m = r == 0 ? l : in.z[r - 1];
      const float2 pn = r == E - 1 ? q : in.z[r + 1];
      const float2 ym = r == 0 ? yom2 : yo2[r - 1];
      float2 x = fma2(ym, m, fma2(yo2[r], pn, neg2(sub.z[r])));
      if (DL) x = fma2(al2[r], in.z[r], x);
      if (HB) x = fma2(yb2[r], in.z[r], x);
      out.z[r] = fma2(ah2[r], in.z[r], x);
    }
  }
  __device__ __forceinline__ void h1_p(const VecP<E>& in, VecP<E>& out) const {
    float2 l, q;
    l.x = g_up<G>(in.z[E - 1].x);
    l.y = g_up<G>(in.z[E - 1].y);
    q.x = g_down<G>(in.z[0].x);
    q.y = g_down<G>(in.z[0].y);
#pragma unroll
    for (int r = 0; r < E; ++r) {
      const float2 m = r == 0 ? l : in.z[r - 1];
      const float2 pn = r == E - 1 ? q : in.z[r + 1];
      const float om = r == 0 ? (float)h1m : (float)o1[r - 1];
      float2 x = fma2(bc2(om), m, mul2(bc2((float)o1[r]), pn));
      if (HB) x = fma2(bc2((float)d1[r]), in.z[r], x);
      out.z[r] = x;
    }
  }
};

template <int E> struct Log2 { static constexpr int v = E <= 1 ? 0 : 1 + Log2<E / 2>::v; };
template <> struct Log2<1> { static constexpr int v = 0; };

template <typename R, int G_, int E_>
struct OpBitflip {
  static constexpr int G = G_, E = E_, DP_SMEM = 0, SMEM_WORDS = 0;
  static constexpr bool PACKED = false;
  static constexpr bool CN = false;
  static constexpr int ASM_MINB = 1;
  static constexpr int LE = Log2<E>::v, LG = Log2<G>::v, Q = LE + LG;
  R ah[E], al[E];        // 2(H0_ee - c)/rad as hi + lo
  R h[Q > 0 ? Q : 1];
  R yh[Q > 0 ? Q : 1];

  __device__ void load(const R* H, const double*, int d, int lg, void*) {
#pragma unroll
    for (int i = 0; i < Q; ++i) h[i] = H[d + i];
  }
  __device__ void scale(const double* H0d, int d, int lg, const Cheb<R>& ch) {
#pragma unroll
    for (int r = 0; r < E; ++r) split2<R>((H0d[lg * E + r] - ch.cd) * ch.s2d, ah[r], al[r]);
  }
  __device__ __forceinline__ void set_u(R u, const Cheb<R>& ch, int) {
    const R s2 = R(2) * ch.inv_rad;
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
    V t;
#pragma unroll
    for (int r = 0; r < E; ++r) {
      R xr = -sub.re[r], xi = -sub.im[r];
      if (sizeof(R) == 4) { xr = fma(al[r], in.re[r], xr); xi = fma(al[r], in.im[r], xi); }
      t.re[r] = fma(ah[r], in.re[r], xr);
      t.im[r] = fma(ah[r], in.im[r], xi);
    }
    flips(in, t, yh);
    out = t;
  }
  template <class V>
  __device__ __forceinline__ void h1(const V& in, V& out) const {
#pragma unroll
    for (int r = 0; r < E; ++r) { out.re[r] = R(0); out.im[r] = R(0); }
    flips(in, out, h);
  }
};

// Dense H0, H1 staged in shared memory (row-major, padded to DP = G*E): real symmetric (CX = false) as
// {H0_ef, H1_ef} pairs; complex Hermitian (CX = true) as {Re H0_ef, Re H1_ef}, {Im H0_ef, Im H1_ef}
// pair couples, so that (H v)_re = Re H v_re - Im H v_im and (H v)_im = Re H v_im + Im H v_re.  The
// state's elements are broadcast with shuffles.
template <typename R, int G_, int E_, bool CX = false>
struct OpDense {
  static constexpr int G = G_, E = E_, DP = G_ * E_, DP_SMEM = G_ * E_;
  static constexpr int SMEM_WORDS = (CX ? 4 : 2) * DP * DP;   // R words of shared memory
  static constexpr bool PACKED = false;
  static constexpr bool CN = false;
  static constexpr int ASM_MINB = 1;
  using R2 = typename C2<R>::T;
  const R2* Hs;   // shared memory
  int lg;
  R s2h, u2, cs2; // 2/rad, 2u/rad, 2c/rad

  __device__ void load(const R*, const double*, int, int lg_, void* smem) {
    Hs = reinterpret_cast<const R2*>(smem);
    lg = lg_;
  }
  __device__ void scale(const double*, int, int, const Cheb<R>&) {}
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
          if constexpr (CX) {
            const R2 p = Hs[2 * ((lg * E + r) * DP + f)], q = Hs[2 * ((lg * E + r) * DP + f) + 1];
            const R yr = REC ? fma(u2, p.y, s2 * p.x) : p.y;
            const R yi = REC ? fma(u2, q.y, s2 * q.x) : q.y;
            ar[r] = fma(yr, vr, fma(-yi, vi, ar[r]));
            ai[r] = fma(yr, vi, fma(yi, vr, ai[r]));
          } else {
            const R2 p = Hs[(lg * E + r) * DP + f];
            const R y = REC ? fma(u2, p.y, s2 * p.x) : p.y;
            ar[r] = fma(y, vr, ar[r]);
            ai[r] = fma(y, vi, ai[r]);
          }
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
//
// COMP (FP32 propagation): the state is carried as hi + lo.  One sub-step is written as
// v_new = v + Delta with Delta = (a_0 - 1) v + sum_{k>=1} a_k (-i)^k T_k(Y) v, a quantity of size
// ~x|v| whose rounding error is ~eps x |v|; hi + (Delta + lo) is then formed by an error-free
// two-sum.  This cuts the per-step FP32 rounding from ~eps(1+x)|v| to ~eps x |v| (x = tau*rad per
// sub-step).  The coefficients a_0 - 1 (COMP) or a_0 and a_1 enter as hi + lo pairs.
template <bool ADJ, bool COMP, typename R, int E, class Op>
__device__ __forceinline__ void cheb_step(Vec<R, E>& v, Vec<R, E>& lo, const Op& op, const Cheb<R>& ch, int K,
                                          int Sw) {
  for (int s = 0; s < Sw; ++s) {
    const bool on = s < ch.S;   // sub-steps beyond this group's own count are computed and discarded
    Vec<R, E> t0 = v, t1, acc;
    Vec<R, E> zero;
#pragma unroll
    for (int r = 0; r < E; ++r) { zero.re[r] = R(0); zero.im[r] = R(0); }
    op.rec(t0, zero, t1);   // t1 = 2 Y t0
#pragma unroll
    for (int r = 0; r < E; ++r) { t1.re[r] *= R(0.5); t1.im[r] *= R(0.5); }
    // k = 0 (a_0, or a_0 - 1 when compensating) and k = 1 on -i*vector (forward) / +i*vector (adjoint)
    const R sg = ADJ ? R(-1) : R(1);
    const R b0h = COMP ? ch.c0h : ch.a0h, b0l = COMP ? ch.c0l : ch.a0l;
#pragma unroll
    for (int r = 0; r < E; ++r) {
      R xr = fma(sg * ch.a1l, t1.im[r], b0l * t0.re[r]);
      R xi = fma(-sg * ch.a1l, t1.re[r], b0l * t0.im[r]);
      xr = fma(sg * ch.a1h, t1.im[r], xr);
      xi = fma(-sg * ch.a1h, t1.re[r], xi);
      acc.re[r] = fma(b0h, t0.re[r], xr);
      acc.im[r] = fma(b0h, t0.im[r], xi);
    }
    // (t0, t1) = (T_{k-2}, T_{k-1}); each recurrence overwrites the older term in place
    for (int k = 2; k < K; k += 2) {
      op.rec(t1, t0, t0);   // t0 <- T_k
      const R ce = ch.cf[k], cel = ch.cl[k];
#pragma unroll
      for (int r = 0; r < E; ++r) {
        if (sizeof(R) == 4) {
          acc.re[r] = fma(cel, t0.re[r], acc.re[r]);
          acc.im[r] = fma(cel, t0.im[r], acc.im[r]);
        }
        acc.re[r] = fma(ce, t0.re[r], acc.re[r]);
        acc.im[r] = fma(ce, t0.im[r], acc.im[r]);
      }
      if (k + 1 < K) {
        op.rec(t0, t1, t1);   // t1 <- T_{k+1}
        const R co = sg * ch.cf[k + 1], col = sg * ch.cl[k + 1];
#pragma unroll
        for (int r = 0; r < E; ++r) {
          if (sizeof(R) == 4) {
            acc.re[r] = fma(col, t1.im[r], acc.re[r]);
            acc.im[r] = fma(-col, t1.re[r], acc.im[r]);
          }
          acc.re[r] = fma(co, t1.im[r], acc.re[r]);
          acc.im[r] = fma(-co, t1.re[r], acc.im[r]);
        }
      }
    }
#pragma unroll
    for (int r = 0; r < E; ++r) {
      if (!on) continue;
      if (!COMP) {
        v.re[r] = acc.re[r];
        v.im[r] = acc.im[r];
      } else {
        // v_new = v + acc (acc = (a_0 - 1) v + sum_{k>=1}): (hi, lo) <- two_sum(hi, acc + lo)
        const R x = v.re[r], y = v.im[r];
        const R tr = acc.re[r] + lo.re[r], ti = acc.im[r] + lo.im[r];
        const R sr = x + tr, si = y + ti;
        const R br = sr - x, bi = si - y;
        lo.re[r] = (x - (sr - br)) + (tr - br);
        lo.im[r] = (y - (si - bi)) + (ti - bi);
        v.re[r] = sr;
        v.im[r] = si;
      }
    }
  }
}

// exp(-i sgn phi) applied in FP64 to hi + lo, returned as (re, im) doubles per element.
__device__ __forceinline__ void phase_rotate(double cp, double sp, bool adj, double xr, double xi, double& yr, double& yi) {
  if (!adj) { yr = xr * cp + xi * sp; yi = xi * cp - xr * sp; }
  else { yr = xr * cp - xi * sp; yi = xi * cp + xr * sp; }
}

template <bool ADJ, typename R, int E, class Op>
__device__ __forceinline__ void cheb_step(Vec<R, E>& v, const Op& op, const Cheb<R>& ch, int K, int Sw) {
  cheb_step<ADJ, false>(v, v, op, ch, K, Sw);
}

// ------------------------------------------------------------- Crank-Nicolson step (Sec. 3)
// x = (I + i sg h H)^{-1} r (sg = +1: A = I + i tau H/2, sg = -1: B = I - i tau H/2, h = tau/2) by
// Jacobi iterations on the split diag(1 + i sg h H_ee) + off-diagonal: each iteration shrinks the
// error by at most rho = h max_e(|H_{e,e-1}| + |H_{e,e+1}|) (the diagonal has modulus >= 1); the
// caller's K iterations reach rho^K below the working precision (k_cheb_prep).
// FP32 steps (LO): the diagonal quantities repeat at every step, so their FP32 rounding would add up
// over the global trajectories like a small change of tau (a phase drift of ~1e-4 rad over 2 x 10^4
// rotor steps).  Ops with a u-independent diagonal carry t = h H_ee, dr and di as hi + lo pairs
// (th/tl, dr/drl, di/dil, formed in FP64; Op::CN_LO); the others have none.
template <typename R, int E, class Op>
__device__ __forceinline__ void cn_dinv(Vec<R, E>& x, R xr_in[E], R xi_in[E], const Op& op, R sg) {
#pragma unroll
  for (int e = 0; e < E; ++e) {   // x = (dr - i sg di) y
    const R yr = xr_in[e], yi = xi_in[e];
    const R di = sg * op.di[e];
    R xr = di * yi, xi = -di * yr;
    if constexpr (Op::CN_LO) {
      const R dl = sg * op.dil[e];
      xr = fma(op.drl[e], yr, fma(dl, yi, xr));
      xi = fma(op.drl[e], yi, fma(-dl, yr, xi));
    }
    x.re[e] = fma(op.dr[e], yr, xr);
    x.im[e] = fma(op.dr[e], yi, xi);
  }
}

template <typename R, int E, class Op>
__device__ __forceinline__ void cn_solve(Vec<R, E>& x, const Vec<R, E>& r, const Op& op, R h, R sg, int K) {
  // D^{-1} = (1 - i sg h d_e) / (1 + (h d_e)^2) = dr_e - i sg di_e (op.dr, op.di)
  {
    R yr[E], yi[E];
#pragma unroll
    for (int e = 0; e < E; ++e) { yr[e] = r.re[e]; yi[e] = r.im[e]; }
    cn_dinv(x, yr, yi, op, sg);
  }
  for (int k = 1; k < K; ++k) {
    Vec<R, E> o;
    op.template cn_apply<false>(x, o);
    R yr[E], yi[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {   // y = r - i sg h (off x), then x = D^{-1} y
      yr[e] = fma(sg * h, o.im[e], r.re[e]);
      yi[e] = fma(-sg * h, o.re[e], r.im[e]);
    }
    cn_dinv(x, yr, yi, op, sg);
  }
}

// ADJ = false: v <- A^{-1} B v.  ADJ = true: xi <- B^{-1} v, then v <- A xi (= U^H v).  Where
// Op::CN_LO, h H v is formed as (th + tl) v + h (off v); else as h (H v).
template <bool ADJ, typename R, int E, class Op>
__device__ __forceinline__ void cn_step(Vec<R, E>& v, Vec<R, E>& xi, const Op& op, R h, int K) {
  Vec<R, E> o;
  if (!ADJ) {
    op.template cn_apply<!Op::CN_LO>(v, o);
    Vec<R, E> r;
#pragma unroll
    for (int e = 0; e < E; ++e) {   // r = v - i h H v
      r.re[e] = fma(h, o.im[e], v.re[e]);
      r.im[e] = fma(-h, o.re[e], v.im[e]);
      if constexpr (Op::CN_LO) {
        r.re[e] = fma(op.th[e], v.im[e], fma(op.tl[e], v.im[e], r.re[e]));
        r.im[e] = fma(-op.th[e], v.re[e], fma(-op.tl[e], v.re[e], r.im[e]));
      }
    }
    cn_solve(v, r, op, h, R(1), K);
  } else {
    cn_solve(xi, v, op, h, R(-1), K);
    op.template cn_apply<!Op::CN_LO>(xi, o);
#pragma unroll
    for (int e = 0; e < E; ++e) {   // v = xi + i h H xi
      v.re[e] = fma(-h, o.im[e], xi.re[e]);
      v.im[e] = fma(h, o.re[e], xi.im[e]);
      if constexpr (Op::CN_LO) {
        v.re[e] = fma(-op.th[e], xi.im[e], fma(-op.tl[e], xi.im[e], v.re[e]));
        v.im[e] = fma(op.th[e], xi.re[e], fma(op.tl[e], xi.re[e], v.im[e]));
      }
    }
  }
}

// The adjoint of the Crank-Nicolson step propagated FORWARD (the two-trajectory form of a first local
// step): lambda_{j+1} = U_j lambda_j with U_j = A_j^{-1} B_j, and since A_j and B_j commute the
// quantity xi_j = B_j^{-1} lambda_{j+1} that the exact discrete gradient pairs with H1 (psi_j +
// psi_{j+1}) equals A_j^{-1} lambda_j.  So: xi <- A^{-1} v (one solve), then v <- B xi (= U v).
template <typename R, int E, class Op>
__device__ __forceinline__ void cn_step_fwd_xi(Vec<R, E>& v, Vec<R, E>& xi, const Op& op, R h, int K) {
  cn_solve(xi, v, op, h, R(1), K);
  Vec<R, E> o;
  op.template cn_apply<!Op::CN_LO>(xi, o);
#pragma unroll
  for (int e = 0; e < E; ++e) {   // v = xi - i h H xi
    v.re[e] = fma(h, o.im[e], xi.re[e]);
    v.im[e] = fma(-h, o.re[e], xi.im[e]);
    if constexpr (Op::CN_LO) {
      v.re[e] = fma(op.th[e], xi.im[e], fma(op.tl[e], xi.im[e], v.re[e]));
      v.im[e] = fma(-op.th[e], xi.re[e], fma(-op.tl[e], xi.re[e], v.im[e]));
    }
  }
}

// Tridiagonal H with the Crank-Nicolson step of Sec. 3 in place of the Chebyshev series: the same lane
// layout and packed data, but H = H0 + u H1 itself (no centring or scaling).  ah[] holds the H0
// diagonal (scale), cdg/cof the diagonal and the (e, e+1) couplings of H at the current control.
template <typename R, int G_, int E_, bool HB = true>
struct OpTridiagCN : OpTridiag<R, G_, E_, HB> {
  using Base = OpTridiag<R, G_, E_, HB>;
  static constexpr bool CN = true;
  static constexpr bool PACKED = false;
  static constexpr int E = E_, G = G_;
  R cdg[E_], cof[E_], cofm;
  R dr[E_], di[E_];   // inverse of the Jacobi diagonal 1 + i h H_ee: dr - i di (A), dr + i di (B)
  R drl[E_], dil[E_]; // their low parts (CN_LO: u-independent diagonal, FP32 steps)
  R th[E_], tl[E_];   // t = h H_ee as hi + lo (CN_LO)
  static constexpr bool CN_LO = !HB && sizeof(R) == 4;
  R hh;               // tau / 2
  __device__ __forceinline__ void diag_inverse() {
#pragma unroll
    for (int r = 0; r < E_; ++r) {
      const R t = hh * cdg[r];
      dr[r] = R(1) / fma(t, t, R(1));
      di[r] = t * dr[r];
    }
  }
  __device__ void scale(const double* H0d, int d, int lg, const Cheb<R>& ch) {
    hh = ch.h;
#pragma unroll
    for (int r = 0; r < E_; ++r) {
      const int e = lg * E_ + r;
      this->ah[r] = e < d ? (R)H0d[e] : R(0);
      cdg[r] = this->ah[r];
      if constexpr (!HB) {   // the diagonal does not depend on u: coefficients in FP64, as hi + lo
        const double t = e < d ? ch.hd * H0d[e] : 0.0;
        const double den = 1.0 / fma(t, t, 1.0);
        split2<R>(t, th[r], tl[r]);
        split2<R>(den, dr[r], drl[r]);
        split2<R>(t * den, di[r], dil[r]);
      }
    }
  }
  __device__ __forceinline__ void set_u(R u, const Cheb<R>&, int lg) {
#pragma unroll
    for (int r = 0; r < E_; ++r) {
      const int e = this->e0 + r;
      const bool in = e < this->dd;
      const R a = in ? __ldg(this->o0p + e) : R(0);
      const R b = in ? __ldg(this->o1p + e) : R(0);
      cof[r] = a + u * b;
      if constexpr (HB) cdg[r] = fma(u, this->d1[r], this->ah[r]);
    }
    const R t = g_up<G_>(cof[E_ - 1]);
    cofm = lg == 0 ? R(0) : t;
    if constexpr (HB) diag_inverse();
  }
  // out = H in (FULL) or its off-diagonal part alone
  template <bool FULL, class V>
  __device__ __forceinline__ void cn_apply(const V& in, V& out) const {
    R lre = g_up<G_>(in.re[E_ - 1]), lim = g_up<G_>(in.im[E_ - 1]);
    R rre = g_down<G_>(in.re[0]), rim = g_down<G_>(in.im[0]);
#pragma unroll
    for (int r = 0; r < E_; ++r) {
      R mre = r == 0 ? lre : in.re[r - 1], mim = r == 0 ? lim : in.im[r - 1];
      R pre = r == E_ - 1 ? rre : in.re[r + 1], pim = r == E_ - 1 ? rim : in.im[r + 1];
      R om = r == 0 ? cofm : cof[r - 1];
      R xr = fma(om, mre, cof[r] * pre), xi = fma(om, mim, cof[r] * pim);
      if (FULL) { xr = fma(cdg[r], in.re[r], xr); xi = fma(cdg[r], in.im[r], xi); }
      out.re[r] = xr;
      out.im[r] = xi;
    }
  }
};

// Bit-flip H with the Crank-Nicolson step: diagonal H0 (the Jacobi diagonal, independent of u) and
// off-diagonal u H1 = u sum_i h_i X_i.
template <typename R, int G_, int E_>
struct OpBitflipCN : OpBitflip<R, G_, E_> {
  using Base = OpBitflip<R, G_, E_>;
  static constexpr bool CN = true;
  static constexpr int E = E_, G = G_, Q = Base::Q;
  R cdg[E_], dr[E_], di[E_], drl[E_], dil[E_], th[E_], tl[E_], hh;
  static constexpr bool CN_LO = sizeof(R) == 4;
  __device__ void scale(const double* H0d, int d, int lg, const Cheb<R>& ch) {
    hh = ch.h;
#pragma unroll
    for (int r = 0; r < E_; ++r) {   // u-independent diagonal: coefficients in FP64, as hi + lo
      cdg[r] = (R)H0d[lg * E_ + r];
      const double t = ch.hd * H0d[lg * E_ + r];
      const double den = 1.0 / fma(t, t, 1.0);
      split2<R>(t, th[r], tl[r]);
      split2<R>(den, dr[r], drl[r]);
      split2<R>(t * den, di[r], dil[r]);
    }
  }
  __device__ __forceinline__ void set_u(R u, const Cheb<R>&, int) {
#pragma unroll
    for (int i = 0; i < Q; ++i) this->yh[i] = u * this->h[i];
  }
  template <bool FULL, class V>
  __device__ __forceinline__ void cn_apply(const V& in, V& out) const {
    V t;
#pragma unroll
    for (int r = 0; r < E_; ++r) {
      t.re[r] = FULL ? cdg[r] * in.re[r] : R(0);
      t.im[r] = FULL ? cdg[r] * in.im[r] : R(0);
    }
    this->flips(in, t, this->yh);
    out = t;
  }
};

// Dense H with the Crank-Nicolson step: H = H0 + u H1 from the shared-memory pairs; the Jacobi
// diagonal H0_ee + u H1_ee is read from the same pairs.
template <typename R, int G_, int E_>
struct OpDenseCN : OpDense<R, G_, E_> {
  using Base = OpDense<R, G_, E_>;
  static constexpr bool CN = true;
  static constexpr int E = E_, G = G_, DP = Base::DP;
  R cdg[E_], dr[E_], di[E_], hh;
  static constexpr bool CN_LO = false;   // the diagonal depends on u
  __device__ void scale(const double*, int, int, const Cheb<R>& ch) { hh = ch.h; }
  __device__ __forceinline__ void set_u(R u, const Cheb<R>&, int) {
    this->u2 = u;   // mv<true> forms H0_ef + u H1_ef with s2 = 1
#pragma unroll
    for (int r = 0; r < E_; ++r) {
      const int e = this->lg * E_ + r;
      const typename Base::R2 p = this->Hs[e * DP + e];
      cdg[r] = fma(u, p.y, p.x);
      const R t = hh * cdg[r];
      dr[r] = R(1) / fma(t, t, R(1));
      di[r] = t * dr[r];
    }
  }
  template <bool FULL, class V>
  __device__ __forceinline__ void cn_apply(const V& in, V& out) const {
    this->template mv<true>(in, out, R(1));
    if (!FULL) {
#pragma unroll
      for (int r = 0; r < E_; ++r) {
        out.re[r] = fma(-cdg[r], in.re[r], out.re[r]);
        out.im[r] = fma(-cdg[r], in.im[r], out.im[r]);
      }
    }
  }
};

// One time step of the op's scheme on a state (v, lo): the Chebyshev series (compensated when COMP),
// or the Crank-Nicolson step (FP64, lo unused).
template <bool ADJ, bool COMP, typename R, int E, class Op>
__device__ __forceinline__ void prop_step(Vec<R, E>& v, Vec<R, E>& lo, const Op& op, const Cheb<R>& ch, int Kw,
                                          int Sw) {
  if constexpr (Op::CN) {
    Vec<R, E> xi;
    cn_step<ADJ>(v, xi, op, ch.h, Kw);
  } else {
    cheb_step<ADJ, COMP>(v, lo, op, ch, Kw, Sw);
  }
}

// Series coefficients of one sub-interval as packed register pairs (c, c), with the sign of the odd
// terms of the adjoint folded in: the packed step then reads no shared memory and builds no pairs
// inside its term loop.  Valid when the warp's term count is at most KR.
template <int KR>
struct CoefP {
  float2 c[KR], l[KR];   // signed a_k as hi, lo (k >= 2)
  float2 b0h, b0l;       // a_0 (or a_0 - 1 when compensated) as hi, lo
  float2 a1h, a1l;       // signed a_1 as hi, lo
};
template <int KR, bool ADJ, bool COMP>
__device__ __forceinline__ void load_coef(CoefP<KR>& cp, const Cheb<float>& ch) {
  const float sg = ADJ ? -1.f : 1.f;
#pragma unroll
  for (int k = 2; k < KR; ++k) {
    const float s = (k & 1) ? sg : 1.f;
    cp.c[k] = bc2(s * ch.cf[k]);
    cp.l[k] = bc2(s * ch.cl[k]);
  }
  cp.b0h = bc2(COMP ? ch.c0h : ch.a0h);
  cp.b0l = bc2(COMP ? ch.c0l : ch.a0l);
  cp.a1h = bc2(sg * ch.a1h);
  cp.a1l = bc2(sg * ch.a1l);
}

// cheb_step_p with the coefficients in registers (K <= KR terms, warp-uniform).
template <bool COMP, int KR, int E, class Op>
__device__ __forceinline__ void cheb_step_pr(VecP<E>& v, VecP<E>& lo, const Op& op, const CoefP<KR>& cp, int K,
                                             int Sw, int S) {
  for (int s = 0; s < Sw; ++s) {
    const bool on = s < S;
    VecP<E> t0 = v, t1, acc, o, zero;
#pragma unroll
    for (int r = 0; r < E; ++r) zero.z[r] = make_float2(0.f, 0.f);
    op.rec_p(t0, zero, t1);   // t1 = 2 Y t0
#pragma unroll
    for (int r = 0; r < E; ++r) {
      t1.z[r] = mul2(t1.z[r], bc2(0.5f));
      acc.z[r] = fma2(cp.b0h, t0.z[r], mul2(cp.b0l, t0.z[r]));
      o.z[r] = fma2(cp.a1h, t1.z[r], mul2(cp.a1l, t1.z[r]));
    }
#pragma unroll
    for (int k = 2; k < KR; k += 2) {
      if (k >= K) break;
      op.rec_p(t1, t0, t0);   // t0 <- T_k
#pragma unroll
      for (int r = 0; r < E; ++r) acc.z[r] = fma2(cp.c[k], t0.z[r], fma2(cp.l[k], t0.z[r], acc.z[r]));
      if (k + 1 < K && k + 1 < KR) {
        op.rec_p(t0, t1, t1);   // t1 <- T_{k+1}
#pragma unroll
        for (int r = 0; r < E; ++r) o.z[r] = fma2(cp.c[k + 1], t1.z[r], fma2(cp.l[k + 1], t1.z[r], o.z[r]));
      }
    }
#pragma unroll
    for (int r = 0; r < E; ++r) {
      acc.z[r].x += o.z[r].y;
      acc.z[r].y -= o.z[r].x;
    }
    if (!on) continue;
#pragma unroll
    for (int r = 0; r < E; ++r) {
      if (!COMP) {
        v.z[r] = acc.z[r];
      } else {
        const float2 x = v.z[r];
        const float2 t = add2(acc.z[r], lo.z[r]);
        const float2 sm = add2(x, t);
        const float2 bb = add2(sm, neg2(x));
        lo.z[r] = add2(add2(x, neg2(add2(sm, neg2(bb)))), add2(t, neg2(bb)));
        v.z[r] = sm;
      }
    }
  }
}

// cheb_step on packed FP32 states (the same series, sub-steps and compensation).  LOC = false drops
// the low parts of a_k for k >= 2 and DL = false that of the diagonal: both roundings repeat at every
// step, so the global sweeps (tens of thousands of steps) keep them, while the sweeps over one
// sub-interval (the sub-problems: ~10^2 steps) may leave them out at ~10^-8 relative cost.  Odd terms multiply
// (-i)^k (forward) or (+i)^k (adjoint): they are summed into a separate packed accumulator o with
// their signed real coefficients and folded in once per sub-step, acc += (o.im, -o.re), so the
// inner loop has no re/im swaps.
template <bool ADJ, bool COMP, bool LOC = true, bool DL = true, int E, class Op>
__device__ __forceinline__ void cheb_step_p(VecP<E>& v, VecP<E>& lo, const Op& op, const Cheb<float>& ch, int K,
                                            int Sw) {
  for (int s = 0; s < Sw; ++s) {
    const bool on = s < ch.S;
    VecP<E> t0 = v, t1, acc, o, zero;
#pragma unroll
    for (int r = 0; r < E; ++r) zero.z[r] = make_float2(0.f, 0.f);
    op.template rec_p<DL>(t0, zero, t1);   // t1 = 2 Y t0
#pragma unroll
    for (int r = 0; r < E; ++r) t1.z[r] = mul2(t1.z[r], bc2(0.5f));
    const float sg = ADJ ? -1.f : 1.f;
    const float b0h = COMP ? ch.c0h : ch.a0h, b0l = COMP ? ch.c0l : ch.a0l;
#pragma unroll
    for (int r = 0; r < E; ++r) {
      acc.z[r] = fma2(bc2(b0h), t0.z[r], mul2(bc2(b0l), t0.z[r]));
      o.z[r] = fma2(bc2(sg * ch.a1h), t1.z[r], mul2(bc2(sg * ch.a1l), t1.z[r]));
    }
    for (int k = 2; k < K; k += 2) {
      op.template rec_p<DL>(t1, t0, t0);   // t0 <- T_k
      const float2 ce = bc2(ch.cf[k]), cel = bc2(ch.cl[k]);
#pragma unroll
      for (int r = 0; r < E; ++r) acc.z[r] = fma2(ce, t0.z[r], LOC ? fma2(cel, t0.z[r], acc.z[r]) : acc.z[r]);
      if (k + 1 < K) {
        op.template rec_p<DL>(t0, t1, t1);   // t1 <- T_{k+1}
        const float2 co = bc2(sg * ch.cf[k + 1]), col = bc2(sg * ch.cl[k + 1]);
#pragma unroll
        for (int r = 0; r < E; ++r) o.z[r] = fma2(co, t1.z[r], LOC ? fma2(col, t1.z[r], o.z[r]) : o.z[r]);
      }
    }
#pragma unroll
    for (int r = 0; r < E; ++r) {
      acc.z[r].x += o.z[r].y;
      acc.z[r].y -= o.z[r].x;
    }
    if (!on) continue;
#pragma unroll
    for (int r = 0; r < E; ++r) {
      if (!COMP) {
        v.z[r] = acc.z[r];
      } else {
        // (hi, lo) <- two_sum(hi, acc + lo)
        const float2 x = v.z[r];
        const float2 t = add2(acc.z[r], lo.z[r]);
        const float2 sm = add2(x, t);
        const float2 bb = add2(sm, neg2(x));
        lo.z[r] = add2(add2(x, neg2(add2(sm, neg2(bb)))), add2(t, neg2(bb)));
        v.z[r] = sm;
      }
    }
  }
}

// Two packed FP32 states stepped forward together under the same U_j (the two trajectories of a
// sub-problem): the same series, sub-steps and compensation as cheb_step_p, with the recurrences of
// the two states interleaved in one term loop, so that each supplies independent instructions while
// the other waits on its shuffles.
template <bool COMP, bool LOC = true, bool DL = true, int E, class Op>
__device__ __forceinline__ void cheb_step_p2(VecP<E>& v, VecP<E>& lo, VecP<E>& w, VecP<E>& wlo, const Op& op,
                                             const Cheb<float>& ch, int K, int Sw) {
  for (int s = 0; s < Sw; ++s) {
    const bool on = s < ch.S;
    VecP<E> t0 = v, t1, acc, o, q0 = w, q1, bcc, oq, zero;
#pragma unroll
    for (int r = 0; r < E; ++r) zero.z[r] = make_float2(0.f, 0.f);
    op.template rec_p<DL>(t0, zero, t1);
    op.template rec_p<DL>(q0, zero, q1);
#pragma unroll
    for (int r = 0; r < E; ++r) {
      t1.z[r] = mul2(t1.z[r], bc2(0.5f));
      q1.z[r] = mul2(q1.z[r], bc2(0.5f));
    }
    const float b0h = COMP ? ch.c0h : ch.a0h, b0l = COMP ? ch.c0l : ch.a0l;
#pragma unroll
    for (int r = 0; r < E; ++r) {
      acc.z[r] = fma2(bc2(b0h), t0.z[r], mul2(bc2(b0l), t0.z[r]));
      o.z[r] = fma2(bc2(ch.a1h), t1.z[r], mul2(bc2(ch.a1l), t1.z[r]));
      bcc.z[r] = fma2(bc2(b0h), q0.z[r], mul2(bc2(b0l), q0.z[r]));
      oq.z[r] = fma2(bc2(ch.a1h), q1.z[r], mul2(bc2(ch.a1l), q1.z[r]));
    }
    for (int k = 2; k < K; k += 2) {
      op.template rec_p<DL>(t1, t0, t0);
      op.template rec_p<DL>(q1, q0, q0);
      const float2 ce = bc2(ch.cf[k]), cel = bc2(ch.cl[k]);
#pragma unroll
      for (int r = 0; r < E; ++r) {
        acc.z[r] = fma2(ce, t0.z[r], LOC ? fma2(cel, t0.z[r], acc.z[r]) : acc.z[r]);
        bcc.z[r] = fma2(ce, q0.z[r], LOC ? fma2(cel, q0.z[r], bcc.z[r]) : bcc.z[r]);
      }
      if (k + 1 < K) {
        op.template rec_p<DL>(t0, t1, t1);
        op.template rec_p<DL>(q0, q1, q1);
        const float2 co = bc2(ch.cf[k + 1]), col = bc2(ch.cl[k + 1]);
#pragma unroll
        for (int r = 0; r < E; ++r) {
          o.z[r] = fma2(co, t1.z[r], LOC ? fma2(col, t1.z[r], o.z[r]) : o.z[r]);
          oq.z[r] = fma2(co, q1.z[r], LOC ? fma2(col, q1.z[r], oq.z[r]) : oq.z[r]);
        }
      }
    }
#pragma unroll
    for (int r = 0; r < E; ++r) {
      acc.z[r].x += o.z[r].y;
      acc.z[r].y -= o.z[r].x;
      bcc.z[r].x += oq.z[r].y;
      bcc.z[r].y -= oq.z[r].x;
    }
    if (!on) continue;
#pragma unroll
    for (int r = 0; r < E; ++r) {
      if (!COMP) {
        v.z[r] = acc.z[r];
        w.z[r] = bcc.z[r];
      } else {
        float2 x = v.z[r], t = add2(acc.z[r], lo.z[r]), sm = add2(x, t), bb = add2(sm, neg2(x));
        lo.z[r] = add2(add2(x, neg2(add2(sm, neg2(bb)))), add2(t, neg2(bb)));
        v.z[r] = sm;
        x = w.z[r]; t = add2(bcc.z[r], wlo.z[r]); sm = add2(x, t); bb = add2(sm, neg2(x));
        wlo.z[r] = add2(add2(x, neg2(add2(sm, neg2(bb)))), add2(t, neg2(bb)));
        w.z[r] = sm;
      }
    }
  }
}

// cheb_step_p2 with the coefficients in registers (forward, K <= KR terms, warp-uniform).
template <bool COMP, bool LOC, bool DL, int KR, int E, class Op>
__device__ __forceinline__ void cheb_step_pr2(VecP<E>& v, VecP<E>& lo, VecP<E>& w, VecP<E>& wlo, const Op& op,
                                              const CoefP<KR>& cp, int K, int Sw, int S) {
  for (int s = 0; s < Sw; ++s) {
    const bool on = s < S;
    VecP<E> t0 = v, t1, acc, o, q0 = w, q1, bcc, oq, zero;
#pragma unroll
    for (int r = 0; r < E; ++r) zero.z[r] = make_float2(0.f, 0.f);
    op.template rec_p<DL>(t0, zero, t1);
    op.template rec_p<DL>(q0, zero, q1);
#pragma unroll
    for (int r = 0; r < E; ++r) {
      t1.z[r] = mul2(t1.z[r], bc2(0.5f));
      q1.z[r] = mul2(q1.z[r], bc2(0.5f));
      acc.z[r] = fma2(cp.b0h, t0.z[r], mul2(cp.b0l, t0.z[r]));
      o.z[r] = fma2(cp.a1h, t1.z[r], mul2(cp.a1l, t1.z[r]));
      bcc.z[r] = fma2(cp.b0h, q0.z[r], mul2(cp.b0l, q0.z[r]));
      oq.z[r] = fma2(cp.a1h, q1.z[r], mul2(cp.a1l, q1.z[r]));
    }
#pragma unroll
    for (int k = 2; k < KR; k += 2) {
      if (k >= K) break;
      op.template rec_p<DL>(t1, t0, t0);
      op.template rec_p<DL>(q1, q0, q0);
#pragma unroll
      for (int r = 0; r < E; ++r) {
        acc.z[r] = fma2(cp.c[k], t0.z[r], LOC ? fma2(cp.l[k], t0.z[r], acc.z[r]) : acc.z[r]);
        bcc.z[r] = fma2(cp.c[k], q0.z[r], LOC ? fma2(cp.l[k], q0.z[r], bcc.z[r]) : bcc.z[r]);
      }
      if (k + 1 < K && k + 1 < KR) {
        op.template rec_p<DL>(t0, t1, t1);
        op.template rec_p<DL>(q0, q1, q1);
#pragma unroll
        for (int r = 0; r < E; ++r) {
          o.z[r] = fma2(cp.c[k + 1], t1.z[r], LOC ? fma2(cp.l[k + 1], t1.z[r], o.z[r]) : o.z[r]);
          oq.z[r] = fma2(cp.c[k + 1], q1.z[r], LOC ? fma2(cp.l[k + 1], q1.z[r], oq.z[r]) : oq.z[r]);
        }
      }
    }
#pragma unroll
    for (int r = 0; r < E; ++r) {
      acc.z[r].x += o.z[r].y;
      acc.z[r].y -= o.z[r].x;
      bcc.z[r].x += oq.z[r].y;
      bcc.z[r].y -= oq.z[r].x;
    }
    if (!on) continue;
#pragma unroll
    for (int r = 0; r < E; ++r) {
      if (!COMP) {
        v.z[r] = acc.z[r];
        w.z[r] = bcc.z[r];
      } else {
        float2 x = v.z[r], t = add2(acc.z[r], lo.z[r]), sm = add2(x, t), bb = add2(sm, neg2(x));
        lo.z[r] = add2(add2(x, neg2(add2(sm, neg2(bb)))), add2(t, neg2(bb)));
        v.z[r] = sm;
        x = w.z[r]; t = add2(bcc.z[r], wlo.z[r]); sm = add2(x, t); bb = add2(sm, neg2(x));
        wlo.z[r] = add2(add2(x, neg2(add2(sm, neg2(bb)))), add2(t, neg2(bb)));
        w.z[r] = sm;
      }
    }
  }
}

}  // namespace ism
