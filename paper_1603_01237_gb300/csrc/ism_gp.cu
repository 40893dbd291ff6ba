// ism_gp.cu -- the Gross-Pitaevskii (condensate) variant of the ISM hot path (Sec. 4, condensates).
//
// Model: i d/dt psi = (-1/2 d^2/dx^2 + V(x, u) + g |psi|^2) psi on a periodic grid of n points,
// V = (x - u)^2 / 2 (harmonic trap, control-shifted centre) or the double well of Sec. 4 (control
// lambda = u, separation D: V = (|x| - u D/2)^2/2 for |x| > u D/4, ((u D)^2/8 - x^2)/2 otherwise),
// J = Re<psi(T)|psi_f>, <a|b> = sum conj(a) b dx.  Time step (Strang, Eq. (OS)):
// psi_{j+1} = K exp(-i tau theta_j) K psi_j with K = F^-1 diag(exp(-i tau k^2/4)) F and
// theta_j = V(x, u_j) + g |K psi_j|^2.
//
// Representation: the sweeps carry a_j = K psi_j, so a step is one pointwise phase and one FFT pair,
//   a_{j+1} = F^-1 [exp(-i tau k^2/2) F (exp(-i tau theta_j) a_j)].
// The adjoint (reverse mode of the discrete map, dJ = Re<lambda_j|d psi_j>) carries nu_j = K^H lambda_j:
//   mu_j = exp(+i tau theta_j) nu_{j+1},   w_j = mu_j + 2 tau g Im(conj(mu_j) a_j) a_j,
//   nu_j = F^-1 [exp(+i tau k^2/2) F w_j],  dJ/du_j = tau sum_k dV/du(x_k) Im(conj(mu_j) a_j)_k dx,
// with lambda_Nt = psi_f.  psi_j = K^H a_j and lambda_j = K nu_j are formed only where stored.
//
// One CTA of max(n/8, 32) threads per state; the FFT is a radix-8 Stockham transform in shared memory
// (element m at a swizzled position), its twiddles and the kinetic factors computed once per plan in
// FP64 and held as hi + lo (FP32 pairs in mixed precision) in a global table.  Phase factors applied
// at every step are held as (factor - 1) and applied as v + (factor - 1) v, so their rounding is
// relative to the change.
//   k_gp_forward   full forward sweep: psi(t_n) at the partition, a_j for every step, J and F;
//   k_gp_adjoint   full adjoint sweep: chi(t_n) = lambda_{j_n}, the sub-problem targets;
//   k_gp_sub       all sub-problems at once (grid N x B): forward from psi(t_n) storing a_j (skipped in
//                  a first local step, whose trajectories the forward sweep stored), adjoint from
//                  chi(t_{n+1}), gradient of J_n = Re<psi_n(t_{n+1})|chi(t_{n+1})>, ascent step.
#include <cmath>

#include "ism_device.cuh"
#include "ism_gp.h"
#include "ism_launch.h"

namespace ism {
namespace {

template <typename T> __device__ __forceinline__ T cmul(T a, T b) {
  T c;
  c.x = a.x * b.x - a.y * b.y;
  c.y = a.x * b.y + a.y * b.x;
  return c;
}
template <typename T> __device__ __forceinline__ T cadd(T a, T b) { T c; c.x = a.x + b.x; c.y = a.y + b.y; return c; }
template <typename T> __device__ __forceinline__ T csub(T a, T b) { T c; c.x = a.x - b.x; c.y = a.y - b.y; return c; }
template <typename T> __device__ __forceinline__ T cconj(T a) { a.y = -a.y; return a; }
// a * (bh + bl) for a factor b held as hi + lo: every transform applies the same rounded twiddles and
// kinetic factors at every step, so their FP32 rounding would add up over the steps like a bias.
template <typename T> __device__ __forceinline__ T cmul_hl(T a, T bh, T bl) {
  T c;
  c.x = fma(a.x, bh.x, fma(-a.y, bh.y, fma(a.x, bl.x, -a.y * bl.y)));
  c.y = fma(a.x, bh.y, fma(a.y, bh.x, fma(a.x, bl.y, a.y * bl.x)));
  return c;
}

__device__ __forceinline__ void sc(float x, float& s, float& c) { sincosf(x, &s, &c); }
__device__ __forceinline__ void sc(double x, double& s, double& c) { sincos(x, &s, &c); }

// exp(i phi) - 1 = -2 sin^2(phi/2) + 2i sin(phi/2) cos(phi/2): one sine-cosine pair of the half
// angle, without cancellation for small phi
template <typename T, typename R> __device__ __forceinline__ T expm1i(R phi) {
  R s, c;
  sc(R(0.5) * phi, s, c);
  T e;
  e.x = R(-2) * s * s;
  e.y = R(2) * s * c;
  return e;
}

// 4-point DFT: X_k = sum_r a_r exp(-+ 2 pi i r k / 4)
template <typename T, bool INV>
__device__ __forceinline__ void dft4(T& a0, T& a1, T& a2, T& a3) {
  T c0 = cadd(a0, a2), c1 = csub(a0, a2), c2 = cadd(a1, a3), d = csub(a1, a3);
  T c3;   // (-i)(a1 - a3) forward, (+i)(a1 - a3) inverse
  if (!INV) { c3.x = d.y; c3.y = -d.x; } else { c3.x = -d.y; c3.y = d.x; }
  a0 = cadd(c0, c2);
  a2 = csub(c0, c2);
  a1 = cadd(c1, c3);
  a3 = csub(c1, c3);
}

// 8-point DFT in registers: X_{2m} = DFT4(v_r + v_{r+4}), X_{2m+1} = DFT4(w^r (v_r - v_{r+4})),
// w = exp(-+ i pi / 4)
template <typename R, bool INV>
__device__ __forceinline__ void dft8(typename C2<R>::T* v) {
  using T = typename C2<R>::T;
  constexpr double hd = 0.70710678118654752440;
  const R h = (R)hd, hl = (R)(hd - (double)(R)hd);   // 1/sqrt(2) as hi + lo (lo = 0 in FP64)
  T a[4], b[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) { a[r] = cadd(v[r], v[r + 4]); b[r] = csub(v[r], v[r + 4]); }
  {   // w^1 = (1 -+ i)/sqrt(2)
    const T t = b[1];
    const R p = t.x + t.y, m = t.y - t.x, q = t.x - t.y;
    if (!INV) { b[1].x = fma(h, p, hl * p); b[1].y = fma(h, m, hl * m); }
    else { b[1].x = fma(h, q, hl * q); b[1].y = fma(h, p, hl * p); }
  }
  {   // w^2 = -+ i
    const T t = b[2];
    if (!INV) { b[2].x = t.y; b[2].y = -t.x; } else { b[2].x = -t.y; b[2].y = t.x; }
  }
  {   // w^3 = (-1 -+ i)/sqrt(2)
    const T t = b[3];
    const R p = t.x + t.y, m = t.y - t.x, q = t.x - t.y;
    if (!INV) { b[3].x = fma(h, m, hl * m); b[3].y = -fma(h, p, hl * p); }
    else { b[3].x = -fma(h, p, hl * p); b[3].y = fma(h, q, hl * q); }
  }
  dft4<T, INV>(a[0], a[1], a[2], a[3]);
  dft4<T, INV>(b[0], b[1], b[2], b[3]);
#pragma unroll
  for (int m = 0; m < 4; ++m) { v[2 * m] = a[m]; v[2 * m + 1] = b[m]; }
}

// Shared-memory position of state element m: its low four index bits XORed with bits 3..6 (a
// permutation of every aligned block of 128 elements, so buffers keep their size).  The Stockham
// stores of the first two radix-8 passes go to strides of 8 and 64 elements, which fall on the same
// banks unswizzled (up to 8 wavefronts per 8-byte warp access); swizzled, every load and store of the
// transform and every element-wise loop over m takes the minimum of two.
__device__ __forceinline__ int sw(int m) { return m ^ ((m >> 3) & 15); }

struct Ident {
  template <class T> __device__ __forceinline__ T operator()(int, int, T v) const { return v; }
  template <class T> __device__ __forceinline__ T operator()(int, T v) const { return v; }
};
struct NoOp {
  __device__ __forceinline__ void operator()() const {}
};

// Stockham radix-8 FFT (unnormalised) of length n = 8^P from x, using y as the other buffer; twiddle
// table W[m] + Wl[m] = exp(-2 pi i m / n) (hi + lo).  Every thread of the block calls it; threads
// t < n/8 compute.
// pre(m, r, v) is applied to every input element as the first pass loads it (thread t loads elements
// m = t + r n/8, r = 0..7), post(m, v) to every output element as the last pass stores it, so
// pointwise factors cost no pass and no barrier of their own.  mid() runs once, after the first
// pass has applied pre (a caller's loads for the next step start there, in registers pre has freed).
// Returns the buffer that holds the result.
template <typename R, bool INV, class Pre = Ident, class Post = Ident, class Mid = NoOp>
__device__ typename C2<R>::T* fft8(typename C2<R>::T* x, typename C2<R>::T* y, const typename C2<R>::T* W,
                                   const typename C2<R>::T* Wl, int n, const Pre& pre = Pre(),
                                   const Post& post = Post(), const Mid& mid = Mid()) {
  using T = typename C2<R>::T;
  const int t = threadIdx.x, q = n >> 3;
  for (int Ns = 1; Ns < n; Ns <<= 3) {
    if (t < q) {
      const int k = t % Ns;
      T v[8];
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const int m = t + r * q;
        v[r] = Ns == 1 ? pre(m, r, x[sw(m)]) : x[sw(m)];
      }
      if (Ns > 1) {   // the first pass's twiddles are all 1
        const int step = n / (Ns << 3);
#pragma unroll
        for (int r = 1; r < 8; ++r) {
          const int i = (k * r * step) & (n - 1);
          T w = W[i], wl = Wl[i];
          if (INV) { w = cconj(w); wl = cconj(wl); }
          v[r] = cmul_hl(v[r], w, wl);
        }
      }
      dft8<R, INV>(v);
      const int base = (t / Ns) * (Ns << 3) + k;
      const bool last = (Ns << 3) == n;
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const int m = base + r * Ns;
        y[sw(m)] = last ? post(m, v[r]) : v[r];
      }
    }
    if (Ns == 1) mid();
    __syncthreads();
    T* tmp = x;
    x = y;
    y = tmp;
  }
  return x;
}

// The per-plan tables of the grid model (n, L, tau and x_min fixed by the plan): twiddles
// exp(-2 pi i m / n), the kinetic factors exp(-i tau k^2/2) - 1 and exp(-i tau k^2/4), each as hi + lo,
// and the grid points x_m as hi + lo.  Layout in units of complex R: W, D2m1, DH, Wl, D2l, DHl
// (n each), then X, Xl (n reals each): 7 n complex R.  Computed once per plan (k_gp_tables) and read
// by every CTA through the L1 cache, so that a CTA's shared memory holds only its three state buffers
// and more CTAs share an SM.
template <typename R>
__device__ void gp_fill_tables(const GPParams& p, typename C2<R>::T* tab) {
  using T = typename C2<R>::T;
  const int n = p.n;
  const double tau = p.tau;
  T *W = tab, *D2m1 = tab + n, *DH = tab + 2 * n, *Wl = tab + 3 * n, *D2l = tab + 4 * n, *DHl = tab + 5 * n;
  R* X = reinterpret_cast<R*>(tab + 6 * n);
  R* Xl = X + n;
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < n; m += gridDim.x * blockDim.x) {
    double s, co;
    sincospi(-2.0 * (double)m / (double)n, &s, &co);
    T w, wl;
    w.x = (R)co;
    w.y = (R)s;
    wl.x = (R)(co - (double)w.x);
    wl.y = (R)(s - (double)w.y);
    W[m] = w;
    Wl[m] = wl;
    const int kk = m < n / 2 ? m : m - n;   // frequency ordering of an unshifted FFT
    const double k = 2.0 * M_PI * (double)kk / p.L;
    const double ph2 = -0.5 * tau * k * k, ph4 = -0.25 * tau * k * k;
    const double h = sin(0.5 * ph2);
    T d, dl;
    const double dx_ = -2.0 * h * h, dy_ = sin(ph2);
    d.x = (R)dx_;
    d.y = (R)dy_;
    dl.x = (R)(dx_ - (double)d.x);
    dl.y = (R)(dy_ - (double)d.y);
    D2m1[m] = d;
    D2l[m] = dl;
    double s4, c4;
    sincos(ph4, &s4, &c4);
    T e, el;
    e.x = (R)c4;
    e.y = (R)s4;
    el.x = (R)(c4 - (double)e.x);
    el.y = (R)(s4 - (double)e.y);
    DH[m] = e;
    DHl[m] = el;
    const double xm = p.xmin + m * p.dx;
    X[m] = (R)xm;
    Xl[m] = (R)(xm - (double)X[m]);
  }
}

// This thread's 8 first-pass elements of a stored row (threads beyond n/8 load nothing).
template <typename T> __device__ __forceinline__ void ld_row8(T (&a)[8], const T* row, int n) {
  const int t = threadIdx.x, q = n >> 3;
  if (t < q) {
#pragma unroll
    for (int r = 0; r < 8; ++r) a[r] = row[t + r * q];
  }
}

template <typename R>
struct GP {
  using T = typename C2<R>::T;
  T *A, *B, *C;                   // state, scratch, spare (shared memory)
  const T *W, *D2m1, *DH;         // twiddles, exp(-i tau k^2/2)-1, exp(-i tau k^2/4) (per-plan table)
  const T *Wl, *D2l, *DHl;        // low parts of the three tables (zero in FP64)
  const R *X, *Xl;                // grid points x_m as hi + lo
  int n;
  double dx, tau, g, xmin;
  int pot;            // 0 harmonic, 1 double well
  R dh, dq, d28;      // D/2, D/4, D^2/8 (double well)
  double* red;

  __device__ void setup(const GPParams& p, unsigned char* smem, double* red_) {
    T* base = reinterpret_cast<T*>(smem);
    const T* tab = reinterpret_cast<const T*>(p.tab);
    n = p.n;
    A = base;
    B = base + n;
    C = base + 2 * n;
    W = tab;
    D2m1 = tab + n;
    DH = tab + 2 * n;
    Wl = tab + 3 * n;
    D2l = tab + 4 * n;
    DHl = tab + 5 * n;
    X = reinterpret_cast<const R*>(tab + 6 * n);
    Xl = X + n;
    dx = p.dx;
    tau = p.tau;
    g = p.g;
    xmin = p.xmin;
    pot = p.pot;
    dh = (R)(0.5 * p.dw);
    dq = (R)(0.25 * p.dw);
    d28 = (R)(0.125 * p.dw * p.dw);
    red = red_;
  }

  // buf <- F^-1 diag(f) F pre(buf) (f = full-step factor, or half-step; conjugated for the adjoint).
  // buf is A or C; B is the scratch of every transform.  The forward transform applies pre on load
  // and f on store, the inverse the 1/n normalisation on store; with 2 log_8(n) passes in all (an
  // even number) the result lands back in buf.
  template <bool ADJ, bool FULL, class Pre = Ident, class Mid = NoOp>
  __device__ void kinetic(T* buf, const Pre& pre = Pre(), const Mid& mid = Mid()) {
    const T* fh = FULL ? D2m1 : DH;
    const T* fl = FULL ? D2l : DHl;
    auto factor = [fh, fl](int m, T v) {
      T f = fh[m], g = fl[m];
      if (ADJ) { f = cconj(f); g = cconj(g); }
      return FULL ? cadd(v, cmul_hl(v, f, g)) : cmul_hl(v, f, g);
    };
    T* X = fft8<R, false>(buf, B, W, Wl, n, pre, factor, mid);
    T* other = (X == buf) ? B : buf;
    const R inv_n = (R)(1.0 / (double)n);
    auto scale = [inv_n](int, T v) {
      v.x *= inv_n;
      v.y *= inv_n;
      return v;
    };
    fft8<R, true>(X, other, W, Wl, n, Ident(), scale);
  }

  // V(x_m, u) and dV/du(x_m, u); x_m = X + Xl (hi + lo)
  __device__ __forceinline__ R pot_v(int m, R u) const {
    if (!pot) {
      const R xm = (X[m] - u) + Xl[m];
      return R(0.5) * xm * xm;
    }
    const R xh = X[m], xl = Xl[m];
    const R axh = fabs(xh), axl = xh < R(0) ? -xl : xl;
    if (axh + axl > u * dq) {
      const R t = (axh - u * dh) + axl;
      return R(0.5) * t * t;
    }
    return R(0.5) * (u * u * d28 - fma(xh, xh, R(2) * xh * xl));
  }
  __device__ __forceinline__ R pot_du(int m, R u) const {
    if (!pot) return (u - X[m]) - Xl[m];
    const R xh = X[m], xl = Xl[m];
    const R axh = fabs(xh), axl = xh < R(0) ? -xl : xl;
    if (axh + axl > u * dq) return -dh * ((axh - u * dh) + axl);
    return u * d28;
  }
  __device__ R theta(int m, R u, T a) const { return pot_v(m, u) + (R)g * (a.x * a.x + a.y * a.y); }

  // One forward Strang step on a = A (a_{j+1} = F^-1 e^{-i tau k^2/2} F e^{-i tau theta} a_j), with
  // the potential factor applied as the first FFT pass loads each element; `keep`, if not null,
  // receives a_j on the way.
  __device__ void step(double u, T* keep) { step_on(A, u, keep); }
  // the same step on buf (A, or C for a recomputed segment)
  __device__ void step_on(T* buf, double u, T* keep) {
    const R ur = (R)u, tr = (R)tau;
    const GP* self = this;
    kinetic<false, true>(buf, [self, ur, tr, keep](int m, int, T a) {
      if (keep) keep[m] = a;
      const T e = expm1i<T, R>(-tr * self->theta(m, ur, a));
      return cadd(a, cmul(e, a));
    });
  }

  // Checkpointed trajectories: a_{c0} .. a_{c1-1} recomputed from the stored a_{c0} (ck) into seg
  // (row i - c0), propagated in the spare buffer C with the same steps as the forward sweep that
  // stored the checkpoint, so every recomputed state equals the one it replaces bit for bit.
  __device__ void recompute(const T* ck, const double* ub, int c0, int c1, T* seg) {
    for (int m = threadIdx.x; m < n; m += blockDim.x) C[sw(m)] = ck[m];
    __syncthreads();
    for (int i = c0; i < c1; ++i) step_on(C, ub[i], seg + (long)(i - c0) * n);
    __syncthreads();
  }

  __device__ double sum(double v) {
    for (int m = 16; m >= 1; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0.0;
    for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) s += red[w];
    __syncthreads();
    return s;
  }

  // adjoint step at a_j (global, complex R, per element): A holds nu_{j+1} on entry and nu_j on exit;
  // the pointwise part runs as the first FFT pass loads each element.  GRAD: also return dJ/du_j
  // (FP64 block sum of FP32 per-thread partials); the global adjoint sweep needs only the states.
  // aj[r] = a_j at element t + r n/8 (this thread's elements of the first FFT pass), loaded one step
  // ahead so that the global-memory latency is off the step's critical path: once the first pass has
  // consumed a_j, aj is refilled from next_row (a_{j-1}; null: left as is) while the remaining five
  // passes run.
  template <bool GRAD>
  __device__ double adjoint_step(T (&aj)[8], double u, const T* next_row) {
    const R ur = (R)u, tr = (R)tau, f2 = R(2) * (R)tau * (R)g;
    R part = R(0);
    const GP* self = this;
    kinetic<true, true>(A, [self, &aj, ur, tr, f2, &part](int m, int r, T nu) {
      const T a = aj[r];
      const T e = expm1i<T, R>(tr * self->theta(m, ur, a));
      const T mu = cadd(nu, cmul(e, nu));
      const R im = mu.x * a.y - mu.y * a.x;   // Im(conj(mu) a)
      if (GRAD) part = fma(self->pot_du(m, ur), im, part);
      T w;
      const R f = f2 * im;
      w.x = mu.x + f * a.x;
      w.y = mu.y + f * a.y;
      return w;
    }, [&aj, next_row, self] {
      if (next_row) ld_row8(aj, next_row, self->n);
    });
    if (!GRAD) return 0.0;
    return tau * dx * sum((double)part);
  }
};


// Resident CTAs per SM an FP32 sweep is compiled for (64 threads each at n = 512).  Each FP32 kernel
// comes twice: unbounded (TP = false), where the compiler spends up to 255 registers on the unrolled
// transforms -- the shortest step, four CTAs per SM -- for launches that fill no more than that; and
// bounded (TP = true) for batches: ten CTAs per SM for the sequential sweeps (one CTA per problem,
// 1520 problems in one wave on 152 SMs), eight for the sub-problems.  FP64 is never bounded.
template <typename R, bool TP> constexpr int gp_min_ctas(int fp32) { return TP && sizeof(R) == 4 ? fp32 : 1; }
constexpr long GP_TP_MIN_CTAS = 4L * 152;   // CTAs of a launch from which the bounded kernels run

template <typename R> __device__ __forceinline__ typename C2<R>::T ld_state(const double2* src, int m) {
  typename C2<R>::T v;
  const double2 z = src[m];
  v.x = (R)z.x;
  v.y = (R)z.y;
  return v;
}

// ------------------------------------------------------------------------------------ kernels
template <typename R, bool TP>
__global__ void __launch_bounds__(64, (gp_min_ctas<R, TP>(10))) k_gp_forward(GPParams p) {
  using T = typename C2<R>::T;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ double red[32];
  GP<R> s;
  s.setup(p, smem, red);
  const int b = blockIdx.x, n = p.n;
  const double* ub = p.u + (long)b * p.Nt;
  // the whole trajectory (cks == 0), or a_j at the checkpoints j = j_n + k cks of every sub-interval
  T* traj = p.cks ? nullptr : reinterpret_cast<T*>(p.traj) + (long)b * (p.Nt + 1) * n;
  T* gck = p.cks ? reinterpret_cast<T*>(p.gck) + (long)b * p.N * p.nck * n : nullptr;
  double2* psin = p.psin + (long)b * (p.N + 1) * n;
  for (int m = threadIdx.x; m < n; m += blockDim.x) s.A[sw(m)] = ld_state<R>(p.psi_i, m);
  __syncthreads();
  s.kinetic<false, false>(s.A);   // a_0 = K psi_i
  int nn = 0;
  for (int j = 0; j <= p.Nt; ++j) {
    if (nn <= p.N && j == p.jn[nn]) {   // psi(t_n) = K^H a_j, and J, F at the end
      for (int m = threadIdx.x; m < n; m += blockDim.x) s.C[sw(m)] = s.A[sw(m)];
      __syncthreads();
      s.kinetic<true, false>(s.C);   // scratch B; the live state A is untouched
      for (int m = threadIdx.x; m < n; m += blockDim.x) {
        const T v = s.C[sw(m)];
        psin[(long)nn * n + m] = make_double2((double)v.x, (double)v.y);
      }
      if (j == p.Nt) {
        double orr = 0.0, oi = 0.0;
        for (int m = threadIdx.x; m < n; m += blockDim.x) {
          const T v = s.C[sw(m)];
          const double2 f = p.psi_f[m];
          orr += (double)v.x * f.x + (double)v.y * f.y;
          oi += (double)v.x * f.y - (double)v.y * f.x;
        }
        orr = s.sum(orr) * p.dx;
        oi = s.sum(oi) * p.dx;
        if (threadIdx.x == 0) {
          if (!isfinite(orr) || !isfinite(oi)) atomicOr(p.status, ST_NONFINITE);
          p.J[b] = orr;
          p.F[b] = orr * orr + oi * oi;
          if (p.Jhist) p.Jhist[(long)b * p.hist_stride + p.hist_k] = orr;
        }
      }
      ++nn;
      __syncthreads();
    }
    if (j == p.Nt) break;
    T* keep = traj ? traj + (long)j * n : nullptr;   // a_j is stored as the step reads it
    if (gck) {
      const int o = j - p.jn[nn - 1];                // step j lies in sub-interval nn - 1
      if (o % p.cks == 0) keep = gck + ((long)(nn - 1) * p.nck + o / p.cks) * n;
    }
    s.step(ub[j], keep);
  }
  if (p.count && threadIdx.x == 0) atomicAdd(p.count, (unsigned long long)p.Nt);
}

template <typename R, bool TP>
__global__ void __launch_bounds__(64, (gp_min_ctas<R, TP>(10))) k_gp_adjoint(GPParams p) {
  using T = typename C2<R>::T;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ double red[32];
  GP<R> s;
  s.setup(p, smem, red);
  const int b = blockIdx.x, n = p.n;
  const double* ub = p.u + (long)b * p.Nt;
  const T* traj = p.cks ? nullptr : reinterpret_cast<const T*>(p.traj) + (long)b * (p.Nt + 1) * n;
  const T* gck = p.cks ? reinterpret_cast<const T*>(p.gck) + (long)b * p.N * p.nck * n : nullptr;
  T* seg = p.cks ? reinterpret_cast<T*>(p.segb) + (long)b * p.N * p.cks * n : nullptr;
  double2* chin = p.chin + (long)b * (p.N + 1) * n;
  for (int m = threadIdx.x; m < n; m += blockDim.x) {
    s.A[sw(m)] = ld_state<R>(p.psi_f, m);
    chin[(long)p.N * n + m] = p.psi_f[m];
  }
  __syncthreads();
  s.kinetic<true, false>(s.A);   // nu_Nt = K^H psi_f
  int nn = p.N - 1;
  T acur[8];
  int c0 = p.Nt;                 // first step of the recomputed segment (checkpointed trajectories)
  if (traj) ld_row8(acur, traj + (long)(p.Nt - 1) * n, n);
  for (int j = p.Nt - 1; j >= 0; --j) {
    const T* next_row = nullptr;
    if (gck) {
      if (j == c0 - 1) {         // the last step of the previous segment: recompute that segment
        const int jb = p.jn[nn], k = (j - jb) / p.cks;
        c0 = jb + k * p.cks;
        s.recompute(gck + ((long)nn * p.nck + k) * n, ub, c0, j + 1, seg);
        ld_row8(acur, seg + (long)(j - c0) * n, n);
      }
      if (j > c0) next_row = seg + (long)(j - 1 - c0) * n;
    } else if (j > 0) {
      next_row = traj + (long)(j - 1) * n;
    }
    s.template adjoint_step<false>(acur, ub[j], next_row);
    if (nn >= 0 && j == p.jn[nn]) {   // chi(t_n) = lambda_j = K nu_j
      for (int m = threadIdx.x; m < n; m += blockDim.x) s.C[sw(m)] = s.A[sw(m)];
      __syncthreads();
      s.kinetic<false, false>(s.C);   // scratch B; the live state A is untouched
      for (int m = threadIdx.x; m < n; m += blockDim.x) {
        const T v = s.C[sw(m)];
        chin[(long)nn * n + m] = make_double2((double)v.x, (double)v.y);
      }
      --nn;
      __syncthreads();
    }
  }
  if (p.count && threadIdx.x == 0) atomicAdd(p.count, (unsigned long long)p.Nt);
}

// grid (N, B): sub-problem n of problem b
template <typename R, bool TP>
__global__ void __launch_bounds__(64, (gp_min_ctas<R, TP>(8))) k_gp_sub(GPParams p) {
  using T = typename C2<R>::T;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ double red[32];
  GP<R> s;
  s.setup(p, smem, red);
  const int nsub = blockIdx.x, b = blockIdx.y, n = p.n;
  const int j0 = p.jn[nsub], j1 = p.jn[nsub + 1];
  double* ub = p.u + (long)b * p.Nt;
  T* traj = p.cks ? nullptr : reinterpret_cast<T*>(p.traj) + (long)b * (p.Nt + 1) * n;
  T* gck = p.cks ? reinterpret_cast<T*>(p.gck) + ((long)b * p.N + nsub) * p.nck * n : nullptr;
  T* seg = p.cks ? reinterpret_cast<T*>(p.segb) + ((long)b * p.N + nsub) * p.cks * n : nullptr;
  const double2* psin = p.psin + (long)b * (p.N + 1) * n;
  const double2* chin = p.chin + (long)b * (p.N + 1) * n;
  double jr = 0.0;
  if (p.reuse) {
    // first local step: phi_n = psi(t_n) under the same controls, so the sub-problem's trajectory on
    // [t_n, t_{n+1}] is the global forward sweep's -- a_j (or its checkpoints) are already stored, and
    // J_n = Re<psi(t_{n+1})|chi(t_{n+1})> with the stored psi(t_{n+1})
    for (int m = threadIdx.x; m < n; m += blockDim.x) {
      const double2 v = psin[(long)(nsub + 1) * n + m];
      const double2 c = chin[(long)(nsub + 1) * n + m];
      jr += v.x * c.x + v.y * c.y;
    }
  } else {
    // forward from psi(t_n), storing a_j for j0..j1-1 (or every cks-th of them)
    for (int m = threadIdx.x; m < n; m += blockDim.x) s.A[sw(m)] = ld_state<R>(psin + (long)nsub * n, m);
    __syncthreads();
    s.kinetic<false, false>(s.A);
    for (int j = j0; j < j1; ++j) {
      T* keep = traj ? traj + (long)j * n : nullptr;
      if (gck && (j - j0) % p.cks == 0) keep = gck + (long)((j - j0) / p.cks) * n;
      s.step(ub[j], keep);
    }
    // J_n = Re<psi_n(t_{n+1})|chi(t_{n+1})>, psi_n(t_{n+1}) = K^H a_{j1}
    s.kinetic<true, false>(s.A);
    for (int m = threadIdx.x; m < n; m += blockDim.x) {
      const T v = s.A[sw(m)];
      const double2 c = chin[(long)(nsub + 1) * n + m];
      jr += (double)v.x * c.x + (double)v.y * c.y;
    }
  }
  jr = s.sum(jr) * p.dx;
  // adjoint from chi(t_{n+1}): nu_{j1} = K^H chi(t_{n+1})
  for (int m = threadIdx.x; m < n; m += blockDim.x) s.A[sw(m)] = ld_state<R>(chin + (long)(nsub + 1) * n, m);
  __syncthreads();
  s.kinetic<true, false>(s.A);
  double err = 0.0;
  double* gb = p.grad + (long)b * p.Nt;
  T acur[8];
  int c0 = j1;   // first step of the recomputed segment (checkpointed trajectories)
  if (traj) ld_row8(acur, traj + (long)(j1 - 1) * n, n);
  for (int j = j1 - 1; j >= j0; --j) {
    const double uj = ub[j];
    const T* next_row = nullptr;
    if (gck) {
      if (j == c0 - 1) {   // entering a segment at its last step: recompute it (u not yet updated there)
        const int k = (j - j0) / p.cks;
        c0 = j0 + k * p.cks;
        s.recompute(gck + (long)k * n, ub, c0, j + 1, seg);
        ld_row8(acur, seg + (long)(j - c0) * n, n);
      }
      if (j > c0) next_row = seg + (long)(j - 1 - c0) * n;
    } else if (j > j0) {
      next_row = traj + (long)(j - 1) * n;
    }
    const double gj = s.template adjoint_step<true>(acur, uj, next_row);
    err += fabs(gj);
    if (threadIdx.x == 0) {
      gb[j] = gj;
      if (p.update) ub[j] = uj + p.rho * gj / p.tau;
    }
  }
  if (threadIdx.x == 0) {
    const long id = (long)b * p.N + nsub;
    if (p.Jn) p.Jn[id] = jr;
    if (p.err) p.err[id] = err;
    if (p.count) atomicAdd(p.count + 1, (unsigned long long)((p.reuse ? 1 : 2) * (j1 - j0)));
  }
}

template <typename R> size_t gp_smem(int n) { return 3 * (size_t)n * sizeof(typename C2<R>::T); }

template <typename R>
__global__ void k_gp_tables(GPParams p) {
  gp_fill_tables<R>(p, static_cast<typename C2<R>::T*>(const_cast<void*>(p.tab)));
}
int gp_threads(int n) { return n / 8 < 32 ? 32 : n / 8; }

template <typename R, class K>
cudaError_t launch(K kern, const GPParams& p, dim3 grid, cudaStream_t st) {
  const size_t sm = gp_smem<R>(p.n);
  cudaError_t e = raise_smem_cap(reinterpret_cast<const void*>(kern));
  if (e != cudaSuccess) return e;
  kern<<<grid, gp_threads(p.n), sm, st>>>(p);
  return cudaGetLastError();
}

}  // namespace

bool gp_supported(int n) { return n == 64 || n == 512; }   // 8^P points, three states in shared memory

cudaError_t launch_gp_forward(int prec, const GPParams& p, cudaStream_t st) {
  if (prec == 0) return launch<double>(k_gp_forward<double, false>, p, dim3(p.B), st);
  return p.B >= GP_TP_MIN_CTAS ? launch<float>(k_gp_forward<float, true>, p, dim3(p.B), st)
                               : launch<float>(k_gp_forward<float, false>, p, dim3(p.B), st);
}
cudaError_t launch_gp_adjoint(int prec, const GPParams& p, cudaStream_t st) {
  if (prec == 0) return launch<double>(k_gp_adjoint<double, false>, p, dim3(p.B), st);
  return p.B >= GP_TP_MIN_CTAS ? launch<float>(k_gp_adjoint<float, true>, p, dim3(p.B), st)
                               : launch<float>(k_gp_adjoint<float, false>, p, dim3(p.B), st);
}
size_t gp_table_bytes(int prec, int n) { return 7 * (size_t)n * (prec == 0 ? sizeof(double2) : sizeof(float2)); }

cudaError_t launch_gp_tables(int prec, const GPParams& p, cudaStream_t st) {
  const unsigned blocks = (unsigned)((p.n + 127) / 128);
  if (prec == 0) k_gp_tables<double><<<blocks, 128, 0, st>>>(p);
  else k_gp_tables<float><<<blocks, 128, 0, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_gp_sub(int prec, const GPParams& p, cudaStream_t st) {
  if (prec == 0) return launch<double>(k_gp_sub<double, false>, p, dim3(p.N, p.B), st);
  return (long)p.N * p.B >= GP_TP_MIN_CTAS ? launch<float>(k_gp_sub<float, true>, p, dim3(p.N, p.B), st)
                                           : launch<float>(k_gp_sub<float, false>, p, dim3(p.N, p.B), st);
}

}  // namespace ism
