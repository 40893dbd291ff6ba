/*
 * ism.h -- C ABI of the GB300 Intermediate State Method (ISM) library (libism.so).
 *
 * Method: M. K. Riahi, J. Salomon, S. J. Glaser, D. Sugny, "A fully efficient time-parallelized
 * quantum optimal control algorithm" (arXiv:1603.01237).  Section references below are to that paper.
 *
 * Problem (Sec. 2, Eq. (dir)):  i d/dt psi = (H0 + u(t) H1) psi on [0, T], maximise
 *     J[u] = Re<psi(T)|psi_f> - (1/2) int alpha(t) u(t)^2 dt          (ISM_OBJ_OVERLAP)
 * or  J[u] = <psi(T)|O|psi(T)> - (1/2) int alpha(t) u(t)^2 dt         (ISM_OBJ_OBSERVABLE, the
 *     observable variant that Sec. 2 calls a straightforward modification).
 * Discretisation: Nt piecewise-constant steps of tau = T/Nt; step j applies
 *     U_j = exp(-i tau (H0 + u_j H1)).
 * Decomposition (Sec. 2): N sub-intervals with step boundaries j_n = floor(n Nt / N), t_n = j_n tau.
 *
 * Conventions shared by every entry point
 *  - Complex vectors are interleaved (re, im) doubles, element index fastest: a state is 2*d doubles.
 *  - A plan holds `batch` independent control problems that share H0, H1, psi_i, the target, T, Nt, N
 *    and alpha, and differ only in their controls.  Batched arrays are problem-major:
 *    u is [batch][Nt], phi is [batch][N+1][2d], grad is [batch][Nt], Jn is [batch][N].
 *  - Array arguments of the compute calls may be host or device pointers; the library asks the CUDA
 *    runtime which one it is (cudaPointerGetAttributes) and copies host data through its own
 *    device buffers.  The caller owns every array it passes; the plan owns its device scratch and
 *    its CUDA resources and frees them in ism_plan_destroy.
 *  - Every compute call is ordered on the plan's stream and returns after that stream has
 *    finished the call's work, so results in host or device memory are ready on return.
 *  - Errors are returned as ism_status; ism_last_error() gives a message for the calling thread.
 *    No C++ exception crosses the ABI and nothing aborts the process.  Non-finite inputs (or
 *    results) give ISM_ENONFINITE.  A plan must not be used by two threads at once.
 */
#ifndef ISM_H_
#define ISM_H_

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  ISM_OK = 0,
  ISM_EINVAL = 1,          /* bad argument (null pointer, size out of range, inconsistent fields) */
  ISM_ENOMEM = 2,          /* device allocation failed                                          */
  ISM_ECUDA = 3,           /* a CUDA runtime call failed (message in ism_last_error)             */
  ISM_ENONFINITE = 4,      /* NaN/Inf in an input array or in a result                          */
  ISM_ETIMEOUT = 5,        /* a bounded device-side wait gave up                                 */
  ISM_EUNSUPPORTED = 6     /* valid request that this build does not implement                  */
} ism_status;

typedef enum {
  ISM_FP64 = 0,            /* everything in double precision                                    */
  ISM_MIXED = 1            /* propagation in FP32; intermediate states, overlaps, norms,
                              objective and the control update in FP64                          */
} ism_precision;

typedef enum {
  /* H0 and H1 are d x d, row-major: real symmetric, or complex Hermitian with real parts H0, H1
     and imaginary parts ism_problem.H0_imag, H1_imag (antisymmetric).  Sec. 2 states the problem
     for any Hermitian H0, H1; the gradient Im<chi|H1|psi> of Eq. (gradJ) holds unchanged for
     complex H1.  d <= 64: every precision and scheme (complex H: the Chebyshev scheme).
     d = 128 or 256, real symmetric only: the global and sub-interval trajectories are propagated
     as stacked state matrices on the tensor cores (TF32 operands split three ways, FP32
     accumulation), ISM_MIXED and local_iters = 1 only; ism_subinterval_grad is ISM_EUNSUPPORTED. */
  ISM_H_DENSE = 0,
  /* d = 2^q spins.  H0 is diagonal: H0[0..d-1] = diag(H0).  H1 = sum_i h_i X_i (bit flips of
     basis index s, spin i <-> bit i): H1[0..q-1] = h_i.  d <= 1024.  For d <= 64 a state lives in
     part of a warp and the global trajectories go through the assembled sub-interval propagators
     (Sec. 3); for d = 128 .. 1024 a state spans a whole CTA and the global trajectories of
     Algorithm 1 (a)-(b) are propagated directly, step by step.                                   */
  ISM_H_BITFLIP = 1,
  /* H0, H1 symmetric tridiagonal: H[0..d-1] = diagonal, H[d..2d-2] = first off-diagonal
     (H[d+e] couples e and e+1).  d <= 64.                                                        */
  ISM_H_TRIDIAG = 2,
  /* Gross-Pitaevskii condensate (Sec. 4): i d/dt psi = (-1/2 d^2/dx^2 + (x - u)^2/2 + g|psi|^2) psi on a
     periodic grid of d = 64 or 512 points x_k = x_min + k L/d, Strang splitting (Eq. (OS)),
     <a|b> = sum conj(a) b L/d.  H0 = {L, x_min, g}; H1 unused (may be NULL); overlap objective only,
     alpha must be NULL.  The sub-problems are the nonlinear variant of Sec. 4: initial states
     psi(t_n) on the forward trajectory, targets chi(t_n) on the adjoint trajectory (the discrete
     adjoint of the full problem), J_n = Re<psi_n(t_{n+1})|chi(t_{n+1})>, ascent u += rho grad/tau.
     phi arrays of the entry points hold both sets: [batch][2][N+1][2d] = psi(t_n), then chi(t_n). */
  ISM_H_GRID_GP = 3,
  /* The same condensate in the double well of Sec. 4, control lambda = u, separation D > 0:
     V(x, u) = (|x| - u D/2)^2/2 for |x| > u D/4, ((u D)^2/8 - x^2)/2 otherwise (V(x, 0) = x^2/2).
     H0 = {L, x_min, g, D}; everything else as ISM_H_GRID_GP.                                       */
  ISM_H_GRID_GP_DOUBLE_WELL = 4,
  /* Several controls (the five-spin example of Sec. 4, in Liouville space): d = 2^q = 128 .. 1024,
     H(t) = diag(H0) + sum_{c < m} u_c(t) H_c, H_c = sum_b (ax[c][b] X_b + ay[c][b] Y_b) (bit b of the
     basis index; Pauli Y = [[0, -i], [i, 0]]).  H0[0..d-1] = diagonal; H1[(c q + b) 2 + {0, 1}] =
     ax[c][b], ay[c][b] (m = ism_problem.controls, 1..32).  Controls, gradients and the ascent are
     per step and control: every u or grad array of the entry points is [batch][Nt][m].  Overlap
     objective only; alpha must be NULL.                                                           */
  ISM_H_PAULI = 5
} ism_hkind;

typedef enum {
  ISM_OBJ_OVERLAP = 0,     /* J = Re<psi(T)|psi_f>, chi(T) = psi_f (Eq. (adj))                    */
  ISM_OBJ_OBSERVABLE = 1   /* J = <psi(T)|O|psi(T)>, chi(T) = O psi(T), weight 2 on Im-terms      */
} ism_objective;

typedef enum {
  /* exp(-i tau H(u_j)) by the Chebyshev (Jacobi-Anger) series to the truncation threshold cheb_tol:
     the exact piecewise-constant propagator of Eq. (dir) up to rounding; every kind, both precisions */
  ISM_SCHEME_CHEBYSHEV = 0,
  /* the Crank-Nicolson step of Sec. 3: (I + i tau H_j/2) psi_{j+1} = (I - i tau H_j/2) psi_j, the
     linear system solved by Jacobi iterations to cheb_tol (K per step with
     (tau/2)(max off-diagonal row sum of H0 + max|u| that of H1) = rho, rho^K <= cheb_tol; a plan
     whose controls make rho >= 1/2 fails with ISM_EUNSUPPORTED).  The gradients are the exact
     derivatives of this discrete scheme, w (tau/2) Im<xi_j|H1|psi_j + psi_{j+1}> with
     xi_j = (I - i tau H_j/2)^{-1} chi_{j+1}.  Both precisions (ISM_MIXED propagates in FP32, the
     Cayley step being unitary by construction; a u-independent diagonal enters it through FP64
     coefficients split into FP32 hi + lo pairs); the tridiagonal, dense and bit-flip kinds with
     d <= 64 (ISM_EUNSUPPORTED otherwise).                                                         */
  ISM_SCHEME_CRANK_NICOLSON = 1
} ism_scheme;

/* The control problem (Sec. 2).  All pointers are HOST pointers read only during ism_plan. */
typedef struct {
  int d;                   /* Hilbert-space dimension                                            */
  int kind;                /* ism_hkind: packed layout of H0 and H1                               */
  const double* H0;        /* packed per kind (see ism_hkind)                                    */
  const double* H1;        /* packed per kind                                                    */
  const double* psi_i;     /* initial state, 2d interleaved                                       */
  int objective;           /* ism_objective                                                        */
  const double* psi_f;     /* target state, 2d interleaved (ISM_OBJ_OVERLAP)                      */
  const double* O;         /* observable, d x d real symmetric row-major (ISM_OBJ_OBSERVABLE)     */
  double T;                /* control time, > 0                                                   */
  int Nt;                  /* number of piecewise-constant steps, >= 1                            */
  int N;                   /* number of sub-intervals, 1 <= N <= Nt                               */
  const double* alpha;     /* Nt penalty weights alpha_j = alpha(t at step midpoint), or NULL (0)  */
  int batch;               /* independent control problems in the plan, >= 1 (0 is read as 1)    */
  int controls;            /* number of controls m (ISM_H_PAULI; 0 is read as 1, others must be 1) */
  const double* H0_imag;   /* ISM_H_DENSE only: Im H0, d x d antisymmetric row-major, or NULL (0)  */
  const double* H1_imag;   /* ISM_H_DENSE only: Im H1, likewise.  Either non-NULL makes H complex
                              Hermitian (d <= 64, Chebyshev scheme; ISM_EUNSUPPORTED otherwise);
                              an imaginary part that is not antisymmetric is ISM_EINVAL.         */
} ism_problem;

typedef struct {
  int precision;           /* ism_precision                                                        */
  int local_iters;         /* L >= 1 gradient steps per sub-interval per ISM iteration (Alg. 1 (c)) */
  double rho;              /* constant step of the gradient ascent (Eq. (gradStep)), > 0          */
  double cheb_tol;         /* truncation threshold of the Chebyshev series; 0 = default per
                              precision (1e-17 FP64, 1e-10 mixed)                                 */
  int max_spin_iters;      /* iteration cap for device-side waits; 0 = default                    */
  int subproblem_form;     /* gradient of the first local step in ism_iterate:
                              1 = literal sub-problem (psi_n from phi_n, chi_n from phi_{n+1});
                              2 = the two-trajectory form of the proof of Theorem 2 (psi from psi(t_n)
                                  and chi from chi(t_n), both propagated forward, scaled by 1/beta_n;
                                  nothing per step is stored but one overlap): identical at phi = phi^u
                                  in exact arithmetic, and free of the O(1/N) cancellation of
                                  phi_{n+1} - psi_n(t_{n+1}) that FP32 propagation cannot resolve;
                              0 = default: 2 (in FP64 the two forms agree to rounding; 2
                              propagates 2 Nt states per iteration where 1 propagates ~3 Nt).
                              Later local steps (L > 1) and ism_subinterval_grad always use
                              the literal form.                                                  */
  int step1;               /* how Algorithm 1 (a)-(b) obtains psi(t_n), chi(t_n) for d <= 64:
                              1 = propagator assembly and chain (Sec. 3): d Nt state-steps per
                                  problem, parallel over sub-intervals -- lowest latency;
                              2 = direct sweeps: 2 Nt state-steps per problem, sequential in time --
                                  least work, for many problems per plan (the sub-problems then
                                  run the forward and adjoint sweeps of a sub-interval in one
                                  lane group, for throughput, rather than in two concurrent ones);
                              0 = default: 2 when batch >= 96, else 1.  Larger d always sweeps. */
  int scheme;              /* ism_scheme: time step of the piecewise-constant propagation          */
  int ckpt_stride;         /* S, checkpoint stride of the literal sub-problems (every linear kind):
                              the forward sweep of sub-interval n stores psi_n every S steps and
                              the adjoint sweep recomputes each segment of S steps from its stored
                              state, so a sub-problem holds ceil(n_steps / S) states and S vectors
                              instead of its whole trajectory (the first local step in the
                              two-trajectory form propagates psi and chi forward together and
                              stores no states at all).  0 = default, ceil(sqrt(longest
                              sub-interval)); values above the longest sub-interval are clamped.
                              Grid kinds (nonlinear: the adjoint needs every forward state): 0 =
                              the whole forward trajectory is stored (B (Nt+1) d states, the
                              fastest); S > 0 = states every S steps of each sub-interval plus one
                              S-step segment per sub-problem, recomputed forward before its
                              adjoint steps (one more forward propagation per sweep).          */
} ism_options;

typedef struct ism_plan_s* ism_plan_t;

/*
 * ism_plan -- validate a problem, copy it to the device and allocate all scratch.
 *   Defines the partition j_n = floor(n Nt/N), a_n = (T - t_n)/T, b_n = t_n/T (Eq. (cible)),
 *   beta_n = T/(t_{n+1} - t_n) (Theorem 1) and alpha_n = alpha / beta_n (Sec. 2).
 *   cuda_stream: a cudaStream_t (NULL = the legacy default stream) on which all work is ordered.
 *   out: receives the plan handle on ISM_OK, untouched otherwise.
 *   Errors: ISM_EINVAL (sizes, kind/layout mismatch, non-symmetric dense input), ISM_ENONFINITE,
 *   ISM_EUNSUPPORTED (d beyond the kind's limit), ISM_ENOMEM, ISM_ECUDA.
 */
int ism_plan(const ism_problem* prob, const ism_options* opt, void* cuda_stream, ism_plan_t* out);

/* ism_plan_destroy -- free every device buffer of the plan.  NULL is accepted (no-op). */
int ism_plan_destroy(ism_plan_t plan);

/*
 * ism_intermediate_states -- Algorithm 1 steps (a) and (b): the trajectories psi and chi of
 *   Eqs. (dir)/(adj) at the partition times, built through the propagator assembly of Sec. 3
 *   (M_n = prod of U_j over sub-interval n, psi(t_{n+1}) = M_n psi(t_n), chi(t_n) = M_n^H chi(t_{n+1})),
 *   and phi_n = ((T - t_n)/T) psi(t_n) + (t_n/T) chi(t_n) (Eq. (cible)), n = 0..N.
 *   u:   [batch][Nt] controls (host or device).
 *   phi: [batch][N+1][2d] output, FP64 in both precision modes (host or device).
 */
int ism_intermediate_states(ism_plan_t plan, const double* u, double* phi);

/*
 * ism_subinterval_grad -- Algorithm 1 step (c) for one gradient evaluation: for every sub-interval
 *   n and problem, psi_n from psi_n(t_n) = phi_n (Eq. (dirpara)), chi_n backward from
 *   chi_n(t_{n+1}) = phi_{n+1}, and
 *     J_n    = w * (-1/2 ||psi_n(t_{n+1}) - phi_{n+1}||^2) - (tau/2) sum_j (alpha_j/beta_n) u_j^2,
 *     grad_j = w (tau/2) [Im<chi_n|H1|psi_n>(t_{j+1}) + Im<chi_n|H1|psi_n>(t_j)] - tau (alpha_j/beta_n) u_j
 *   (the derivative dJ_n/du_j in the trapezoid reading of the gradient in the proof of Theorem 2;
 *   w = 1 for the overlap objective, 2 for the observable).  beta_n * grad equals the gradient of
 *   J on that sub-interval when phi = phi^u (Theorem 2).
 *   phi:  [batch][N+1][2d] (any states, not only phi^u); u: [batch][Nt];
 *   grad: [batch][Nt] output; Jn: [batch][N] output or NULL.
 */
int ism_subinterval_grad(ism_plan_t plan, const double* phi, const double* u, double* grad, double* Jn);

/*
 * ism_iterate -- run `iters` passes of Algorithm 1 with the constant-step gradient sub-solver:
 *   (a)-(b) as ism_intermediate_states, (c) L = local_iters ascent steps
 *   u_j <- u_j + rho * beta_n * grad_j / tau on each sub-interval with phi fixed (Eq. (gradStep),
 *   read as ascent since J is maximised), (d) the new controls are the concatenation, (e)
 *   Err_k = sum_n sum_j |grad_j| of the first local step.
 *   u_inout:  [batch][Nt] controls, updated in place (host or device).
 *   J_hist:   [batch][iters+1] J[u^(k)] for k = 0..iters, or NULL (then the final objective
 *             evaluation is skipped).
 *   err_hist: [batch][iters] Err_k, or NULL.
 */
int ism_iterate(ism_plan_t plan, int iters, double* u_inout, double* J_hist, double* err_hist);

/*
 * ism_evaluate -- objective at u: J (with penalty) and F = |<psi(T)|psi_f>|^2 (overlap) or
 *   <psi(T)|O|psi(T)> (observable), through the same assembly and chain as (a).
 *   u: [batch][Nt]; J, F: [batch] outputs (host or device), either may be NULL.
 */
int ism_evaluate(ism_plan_t plan, const double* u, double* J, double* F);

/*
 * ism_gradient -- gradient of the full objective J[u] at u (Eq. (gradJ) in its discrete trapezoid
 *   form, penalty included) for every problem of the plan, and J.  By Theorem 2 it is the
 *   concatenation over n of beta_n times the sub-problem gradients at phi = phi^u; the library
 *   evaluates it with the two-trajectory form of the theorem's proof (psi from psi(t_n), chi from
 *   chi(t_{n+1})): one pass of Algorithm 1 (a)-(b) and one parallel sub-interval pass, u unchanged.
 *   For the grid kind it is the reverse-mode gradient of the discrete split-step map.  This is the
 *   backward pass of an automatic-differentiation wrapper around ism_evaluate.
 *   u: [batch][Nt] (host or device); grad: [batch][Nt] output (host or device); J: [batch] or NULL.
 */
int ism_gradient(ism_plan_t plan, const double* u, double* grad, double* J);

/* Work and time accounting of a plan, accumulated over calls until reset.
 *   ms[p], launches[p]: device time (CUDA events around each kernel, only while profiling is on)
 *                       and launches of phase p = 0 assembly, 1 chain, 2 sub-interval.
 *   y_apps[k], terms[k], substeps[k]: for k = 0 assembly, 1 sub-interval sweeps, the number of
 *     applications of the scaled Hamiltonian to one state, of accumulated Chebyshev terms and of
 *     exponential sub-steps -- the algorithmic work from which flop counts follow.
 *   kernels: every kernel the plan launched (the phase kernels and the helpers that check inputs,
 *     refresh propagator parameters and sum Err). */
typedef struct {
  double ms[3];
  long long launches[3];
  unsigned long long y_apps[2];
  unsigned long long terms[2];
  unsigned long long substeps[2];
  long long kernels;
  double norm_drift;        /* largest |norm^2 / reference - 1| of psi(T) and chi(t_0) (the ends of the
                               global trajectories, where it is largest) before the FP64
                               renormalisation of psi(t_n), chi(t_n) (0 for the grid kinds)          */
} ism_stats;

/* ism_set_profiling -- on != 0 records CUDA events around every kernel on the plan's stream. */
int ism_set_profiling(ism_plan_t plan, int on);

/* ism_get_stats -- copy the accumulated accounting into *out (synchronises the plan's stream);
 *   reset != 0 zeroes it afterwards. */
int ism_get_stats(ism_plan_t plan, ism_stats* out, int reset);

/* ism_measure_peak -- the FMA rate this GPU sustains, in TFLOP/s, measured with CUDA events on the
 *   current device: which = 0 packed FP32 FMAs (fma.rn.f32x2, 4 flops each), 1 FP64 FMAs (2 flops).
 *   Every SM runs independent FMA chains for a fixed count; the best of three timed launches after a
 *   warm-up launch.  These are the peaks of the propagation kernels' ALU rooflines (the paper has no
 *   counterpart).  Allocates nothing; ISM_EINVAL for another `which`, ISM_ECUDA on a CUDA error. */
int ism_measure_peak(int which, double* tflops);

/* ism_plan_footprint -- device bytes ism_plan would allocate for (prob, opt), without allocating or
 *   touching a GPU (admission control).  The J/Err history buffers that ism_iterate adds on demand
 *   (16 bytes x batch x (iters + 1)) are not included.  Same validation and errors as ism_plan. */
int ism_plan_footprint(const ism_problem* prob, const ism_options* opt, size_t* bytes);

/* ism_plan_info -- integer facts about a plan, for tests and benchmarks:
 *   key 0: group lanes per state, 1: state elements per lane, 2: kernel launches per ISM
 *   iteration (L = local_iters), 3: bytes of plan-owned device memory, 4: bytes of one stored
 *   sub-interval propagator M_n (0 when none is assembled), 5: 1 when the plan propagates the global
 *   trajectories directly (bit-flip d >= 128, one state per CTA) instead of assembling M_n,
 *   6: how Algorithm 1 (a)-(b) runs (ism_options.step1 after the default is resolved: 1 or 2),
 *   7: tiles per block of the blocked chain (1 = plain chain),
 *   8: the plan's time-step scheme (ism_scheme),
 *   9: lanes per state of the direct sweeps (0 when the plan assembles; fewer lanes with more
 *      elements each once the batch gives every SM two CTAs of that layout),
 *   10: 1 when the plan propagates on the tensor cores (dense d = 128, 256),
 *   11: the checkpoint stride in use (ism_options.ckpt_stride after the default and the clamp are
 *       resolved; grid kinds: 0 when the whole forward trajectory is stored).
 *   Returns -1 for a bad key. */
long long ism_plan_info(ism_plan_t plan, int key);

/*
 * ism_subinterval_grad_noalloc -- the computation of ism_subinterval_grad for callers that cannot
 *   allocate device memory (code inside another framework's memory pool, allocation-free real-time
 *   loops, processes with a device-memory budget fixed up front).  The paper has no counterpart: it
 *   is an addition of this library.  Needs no plan and calls no cudaMalloc, cudaFree or allocating
 *   library routine: all scratch (packed Hamiltonian, partition, penalty weights, status word, the
 *   per-step overlaps and the checkpoints and segment buffer of the literal sub-problem) lives in one
 *   static device array of ISM_NOALLOC_SCRATCH_BYTES that every GPU loading the library holds until
 *   the process exits.  It launches the same kernels as ism_subinterval_grad on a plan of the same
 *   problem and precision, with the default checkpoint stride, and gives the same results bit for bit.
 *   prob:      the problem (host struct and host arrays, as for ism_plan); precision: ism_precision.
 *   phi, u:    [batch][N+1][2d] and [batch][Nt] inputs, DEVICE memory of the current GPU.
 *   grad, Jn:  [batch][Nt] and [batch][N] (Jn may be NULL) outputs, DEVICE memory of the current GPU.
 *   cuda_stream: the stream the work is ordered on.  The call synchronises that stream and reads the
 *   status word back before it returns.  The first call on a device does a one-time set-up: it looks
 *   up the array's device address (cudaGetSymbolAddress) with that device current; make that first
 *   call before any stream capture.  All calls share the array and it keeps the last call's contents
 *   (the status word is cleared on entry); calls whose work overlaps on the GPU race on it.  A problem
 *   needing more scratch than the array holds is rejected with ISM_EINVAL and a message giving both
 *   sizes; host pointers, or device memory of another GPU, for phi, u, grad or Jn give ISM_EINVAL; NaN
 *   or Inf in u or phi gives ISM_ENONFINITE.  Covers the dense (real or complex Hermitian),
 *   tridiagonal and bit-flip kinds with d <= 64 (the Chebyshev step); other kinds and larger d give
 *   ISM_EUNSUPPORTED.  Other errors as ism_subinterval_grad.
 */
#define ISM_NOALLOC_SCRATCH_BYTES (32u << 20)
int ism_subinterval_grad_noalloc(const ism_problem* prob, int precision, const double* phi, const double* u,
                                 double* grad, double* Jn, void* cuda_stream);

/* Message of the last error on the calling thread ("" if none).  Valid until the next call. */
const char* ism_last_error(void);

/* Library version string. */
const char* ism_version(void);

/*
 * Serving loop (no counterpart in the paper, which solves one problem at a time): a server queues
 * submitted solves -- each its own problem, options, initial controls and iteration count, so the
 * Hilbert dimensions, step counts and N of concurrent requests may all differ -- and runs them on
 * `slots` worker threads, one CUDA stream each.  Continuous batching: requests of the structured
 * kinds (tridiagonal, bit-flip) in mixed precision with the Chebyshev step, one local step and one
 * problem each share launches with the other requests of the same (kind, d, N, objective): a worker
 * runs a shared plan of group_capacity rows, one ISM pass over all its active rows at a time, retires
 * the requests that have finished and admits the ones that arrived meanwhile between passes.  Every
 * row is computed independently of the others, so a request's controls and J history are the same,
 * bit for bit, alone and in any mix.  Other requests run on a plan of their own.  A shared plan (or a
 * request's own plan) is admitted when its device footprint fits in what the budget has left; plans
 * stay resident while they run and are released when their last request ends.
 */
typedef struct ism_server_s* ism_server_t;

typedef struct {
  int slots;                 /* concurrent solves (worker threads and CUDA streams), 1..64           */
  size_t hbm_budget_bytes;   /* device memory the admitted plans may hold together                   */
  int group_capacity;        /* rows of a shared plan (continuous batching); 0 = 64; < 0 = no sharing */
  int group_max_steps;       /* step capacity of a shared plan's rows (longer requests open their own
                                group); 0 = 50000                                                    */
} ism_server_options;

enum { ISM_REQ_QUEUED = 0, ISM_REQ_RUNNING = 1, ISM_REQ_DONE = 2, ISM_REQ_FAILED = 3 };

/* ism_server_create -- start the workers on the current CUDA device.  ISM_EINVAL for bad options,
 *   ISM_ENOMEM if the server or its worker threads cannot be created (none is left running). */
int ism_server_create(const ism_server_options* opt, ism_server_t* out);

/* ism_server_submit -- queue a solve: ism_iterate(iters) from u0 ([batch][Nt]) on a plan for (prob,
 *   opt).  Every array of prob and u0 is copied before the call returns.  *id receives the request
 *   id.  Errors: those of ism_plan_footprint; ISM_ENOMEM if the request alone exceeds the budget or
 *   its host copy cannot be allocated.  A plan or solve that fails later, in a worker, is reported by
 *   ism_server_poll with the failing call's status and message. */
int ism_server_submit(ism_server_t srv, const ism_problem* prob, const ism_options* opt, const double* u0,
                      int iters, long long* id);

/* ism_server_poll -- state of a request (ISM_REQ_*); wait != 0 blocks until it is done or failed.
 *   When done, copies the final controls into u_out ([batch][Nt]) and the objective history into
 *   J_hist ([batch][iters+1]) if they are non-NULL; times_ms (3 doubles, may be NULL) receives the
 *   queueing time, the run time and the total latency (-1 while unknown).  Returns the request's
 *   error status if it failed, ISM_EINVAL for an unknown id. */
int ism_server_poll(ism_server_t srv, long long id, int wait, int* state, double* u_out, double* J_hist,
                    double* times_ms);

/* ism_server_release -- forget a finished request (its host copies are freed).  ISM_EINVAL for an
 *   unknown id or a request that is still queued or running. */
int ism_server_release(ism_server_t srv, long long id);

/* ism_server_stats -- out[0] ISM passes run on shared plans, out[1] request-passes they carried (so
 *   out[1] / out[0] requests per shared launch sequence), out[2] the most requests in one pass,
 *   out[3] shared plans opened, out[4] requests run on a plan of their own. */
int ism_server_stats(ism_server_t srv, long long* out);

/* ism_server_destroy -- finish the running solves, fail the queued ones, stop the workers and free
 *   the server.  The caller must make sure that no other call on srv is in progress (in particular
 *   no thread blocked in ism_server_poll with wait != 0) and that none starts afterwards: srv is
 *   freed on return. */
int ism_server_destroy(ism_server_t srv);

#ifdef __cplusplus
}
#endif
#endif /* ISM_H_ */
