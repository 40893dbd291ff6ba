// ism_tc.cu -- the propagation of Algorithm 1 for dense real-symmetric H0, H1 of dimension d = 128 or
// 256 on the tensor cores (tcgen05, TMEM accumulators, TMA-staged operands).
//
// States are stacked as the columns of a real matrix T (d rows; a complex state is two columns, its real
// and imaginary parts).  One Chebyshev term of the step exp(-i tau H(u_j)) (the series of
// ism_device.cuh) needs Y T_k with Y = (H0 + u H1 - c)/rad, and u, c, rad differ from column to column
// (each state has its own control and sub-interval), so the contraction is
//     Z = [H0; H1] T_k      (2d x columns, one GEMM, K = d),
// and the epilogue forms, column by column, T_{k+1} = (2/rad)(Z0 + u Z1) - (2c/rad) T_k - T_{k-1} and the
// series sum.  States of different problems, sub-intervals and directions move in lockstep by step: the
// global sweeps of steps (a)-(b) stack psi forward and chi backward of every problem, the sub-interval
// sweeps of step (c) stack psi_n and chi_n of every (problem, n) in the two-trajectory form of the proof
// of Theorem 2 (both carried forward from psi(t_n), chi(t_n)).
//
// Precision (mixed mode).  The tensor cores take TF32 operands (10-bit mantissa) into FP32 accumulators;
// a single pass would leave ~5e-4 relative error per product.  Every operand is split in two TF32 parts,
// x = x_hi + x_lo (x_lo the TF32 rounding of x - x_hi), and Z = H_hi T_hi + H_hi T_lo + H_lo T_hi: three
// passes, ~2^-22 relative (the dropped H_lo T_lo is below the FP32 rounding of the sums).  The series
// coefficients, 2/rad and 2c/rad enter the epilogue as FP32 hi + lo pairs; the states are carried as
// FP32 hi + lo and updated by an error-free two-sum (v_new = v + Delta), as in the FP32 lane-group
// sweeps; the per-step global phase exp(-i c tau) is applied per segment in FP64.
//
// One CTA owns NS columns (NS/2 states) for the whole sweep (the columns never interact), 1 CTA per SM:
//   warp 0      : TMEM allocation; one elected lane issues the TMA loads of [H0; H1] (hi and lo, in
//                 K-chunks through a two-stage ring) and the tcgen05.mma of every chunk, then commits.
//   warps 1 - 8 : epilogue, two warps per TMEM sub-partition (they split the columns), one thread per
//                 TMEM lane (row f of the output, and f + 128 when d = 256):
//                 reads Z from TMEM, forms T_{k+1} and the series sum, writes T_{k+1} (TF32 hi and lo)
//                 into the shared-memory B operand of the next GEMM and keeps T_k and the sum in TMEM.
// Shared memory: B operand (the CTA's states, K-major, 128-byte swizzle) hi and lo, 64 KB each; two A
// stages of 32 KB.  TMEM (512 columns): Z (2d/128 tiles of NS columns), T_{k-1} and the sum (d/128
// tiles each).
// Every mbarrier wait is bounded; a wait that gives up sets ST_TIMEOUT and an abort flag that every role
// polls, so the CTA winds down, waits (bounded) for its copies and MMAs in flight and frees its TMEM.
#include <cuda.h>   // CUtensorMap and its enums; the encoder is obtained from the runtime

#include <cstdint>
#include <cstring>

#include "ism_kernels.cuh"
#include "ism_launch.h"
#include "ism_tc.h"

namespace ism {
namespace {

// ------------------------------------------------------------------------------- configuration
template <int D>
struct TcCfg {
  static constexpr int NS = 16384 / D;           // real columns per CTA
  static constexpr int NI = NS / 2;              // states per CTA
  static constexpr int MT = 2 * D / 128;         // 128-row tiles of [H0; H1] (and of Z)
  static constexpr int LT = D / 128;             // 128-row tiles of one state
  static constexpr int KC = D == 128 ? 16 : 8;   // K of one A chunk (one TMA stage)
  static constexpr int NCH = D / KC;             // chunks per GEMM
  static constexpr int KSTEPS = KC / 8;          // tcgen05.mma (K = 8 for TF32) per chunk and tile
  static constexpr int ROWB = KC * 4;            // bytes of one A row in a chunk = its swizzle span
  static constexpr int AHALF = 2 * D * ROWB;     // hi (or lo) part of a stage
  static constexpr int STAGE = 2 * AHALF;
  static constexpr int NSTAGE = 2;
  static constexpr int BHALF = NS * D * 4;       // B operand hi (or lo): NS rows of D TF32
  static constexpr int KATOM = NS * 128;         // bytes between the 32-element K atoms of B
  static constexpr int TM_Z = 0, TM_TP = 256, TM_AC = 384;   // TMEM columns of Z, T_{k-1}, series sum
  static constexpr int BOXR = 2 * D < 256 ? 2 * D : 256;     // rows per TMA box
};

constexpr int TC_WARPS = 9;   // warp 0: TMA + MMA; warps 1-8: epilogue (two per TMEM sub-partition)
constexpr int TC_CW = 16;     // columns per epilogue chunk (one 32x32b.x16 TMEM load per operand)
constexpr int TC_THREADS = 32 * TC_WARPS;

// Per-state parameters of the current step, in shared memory.
struct TcPar {
  float ch[KMAX], cl[KMAX];   // signed series coefficients (k = 0: a_0 - 1, k odd: adjoint sign folded in)
  float s2h, s2l, cs2h, cs2l; // 2/rad and 2c/rad as hi + lo
  float u;                    // control of the current step
  int K, S;                   // terms and sub-steps of the current sub-interval
  int n;                      // current sub-interval (global sweeps: moves along the sweep; -1: not set)
  int ln;                     // sub-interval whose parameters are loaded (-1: none)
  int on;                     // the state advances in this step
  double cph, sph;            // segment phase of sub-interval n
  unsigned long long work;    // steps x sub-steps run (accounting)
};

// ---------------------------------------------------------------------------------- PTX helpers
__device__ __forceinline__ float tf32_rn(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// D[tmem] (+)= A[smem] * B[smem]^T (both K-major), TF32 in, FP32 accumulate
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, int acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
      : "memory");
}
// arrive on an mbarrier once every tcgen05.mma issued so far by this thread has completed
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// TC_CW consecutive TMEM columns of this warp's 32 lanes: one register per column
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float (&v)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(taddr),
      "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])),
      "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])),
      "r"(__float_as_uint(v[8])), "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
      "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])), "r"(__float_as_uint(v[15]))
      : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// 2-D tiled TMA load global -> shared, completion counted on `bar`
__device__ __forceinline__ void tma_load_2d(void* dst, const void* tmap, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(tmap), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }

// Shared-memory matrix descriptor of a K-major operand (SM100 format): start address, leading and
// stride byte offsets (16-byte units), version 1, swizzle layout (2: 128 B, 4: 64 B, 6: 32 B).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t sbo, uint32_t layout) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1u << 16;                        // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1u << 46;                        // descriptor version
  d |= (uint64_t)(layout & 7u) << 61;
  return d;
}
// Instruction descriptor of kind::tf32: FP32 accumulator, TF32 A and B, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Byte offset of element (column c, k) of the B operand in its 128-byte-swizzled K-major layout:
// K atoms of 32 elements, NS rows of 128 bytes each, the 16-byte chunk index XORed with row % 8.
template <int D>
__device__ __forceinline__ uint32_t b_off(int c, int k) {
  using C = TcCfg<D>;
  const uint32_t chunk = (uint32_t)((k & 31) >> 2) ^ (uint32_t)(c & 7);
  return (uint32_t)(k >> 5) * C::KATOM + (uint32_t)c * 128u + chunk * 16u + (uint32_t)(k & 3) * 4u;
}

// bounded wait that also gives up once another role has aborted
__device__ __forceinline__ bool tc_wait(uint64_t* bar, unsigned parity, int max_spin, volatile int* abort_flag,
                                        int* status) {
  for (int it = 0; it < max_spin; ++it) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
    if (*abort_flag) return false;
    if (it > 64) __nanosleep(32);
  }
  atomicOr(status, ST_TIMEOUT);
  *abort_flag = 1;
  return false;
}

// ------------------------------------------------------------------------------------ kernel
template <int D>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_tc_sweep(const __grid_constant__ CUtensorMap mhi, const __grid_constant__ CUtensorMap mlo, TcParams p) {
  using C = TcCfg<D>;
  constexpr int NS = C::NS, NI = C::NI;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte alignment of the swizzled operands
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* Bhi = sm;
  unsigned char* Blo = sm + C::BHALF;
  unsigned char* Ast = sm + 2 * C::BHALF;
  TcPar* par = reinterpret_cast<TcPar*>(Ast + C::NSTAGE * C::STAGE);
  float* zred = reinterpret_cast<float*>(par + NI);              // [4 warps][NI/2 pairs][2]
  uint64_t* bars = reinterpret_cast<uint64_t*>(zred + 4 * NI);   // full[2], empty[2], bready, zready
  uint64_t* full = bars;
  uint64_t* empty = bars + 2;
  uint64_t* bready = bars + 4;
  uint64_t* zready = bars + 5;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 6);
  volatile int* cmd = reinterpret_cast<volatile int*>(tmem_slot + 1);
  volatile int* abort_flag = cmd + 1;
  int* kt_st = const_cast<int*>(abort_flag + 1);   // [2]: terms and sub-steps of the current step

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int item0 = blockIdx.x * NI;
  float* vs = p.vstate + (size_t)blockIdx.x * 2 * NS * D;   // [2][NS][D]

  if (threadIdx.x == 0) {
    for (int i = 0; i < 2; ++i) { mbar_init(full + i, 1); mbar_init(empty + i, 1); }
    mbar_init(bready, 1);
    mbar_init(zready, 1);
    *cmd = 0;
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 0) tmem_alloc(tmem_slot, 512);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ======================================================== TMA producer + MMA issuer (one lane)
    if (lane == 0) {
      const uint32_t idesc = idesc_tf32(128, NS);
      const uint32_t alayout = C::ROWB == 64 ? 4u : 6u;   // 64-byte or 32-byte swizzle
      long gc = 0;                                         // chunks loaded so far (stage / phase)
      long gmm = 0;                                        // GEMMs done (bready / zready phase)
      auto load_chunk = [&](long x) -> bool {
        const int st = (int)(x & 1);
        if (x >= 2 && !tc_wait(empty + st, (unsigned)(((x >> 1) - 1) & 1), p.max_spin, abort_flag, p.status)) return false;
        unsigned char* dst = Ast + st * C::STAGE;
        const int k0 = (int)(x % C::NCH) * C::KC;
        mbar_expect_tx(full + st, C::STAGE);
        for (int r = 0; r < 2 * D; r += C::BOXR) {
          tma_load_2d(dst + r * C::ROWB, &mhi, k0, r, full + st);
          tma_load_2d(dst + C::AHALF + r * C::ROWB, &mlo, k0, r, full + st);
        }
        return true;
      };
      bool ok = load_chunk(gc);   // first chunk of the first GEMM, ahead of the epilogue's set-up
      long loaded = ok ? 1 : 0;
      while (ok) {
        if (!tc_wait(bready, (unsigned)(gmm & 1), p.max_spin, abort_flag, p.status)) break;
        if (*cmd == 0) break;
        tc_fence_after();
        for (int c = 0; c < C::NCH && ok; ++c) {
          if (loaded == gc + 1 && !(ok = load_chunk(gc + 1))) break;   // next chunk (of this or the next GEMM)
          if (loaded == gc + 1) ++loaded;
          const int st = (int)(gc & 1);
          if (!(ok = tc_wait(full + st, (unsigned)((gc >> 1) & 1), p.max_spin, abort_flag, p.status))) break;
          tc_fence_after();
          const uint32_t abase = smem_u32(Ast + st * C::STAGE);
#pragma unroll
          for (int ks = 0; ks < C::KSTEPS; ++ks) {
            const int k = c * C::KC + ks * 8;
            const uint32_t boff = (uint32_t)(k >> 5) * C::KATOM + (uint32_t)((k & 31) >> 3) * 32u;
            const uint64_t bh = smem_desc(smem_u32(Bhi) + boff, 1024, 2);
            const uint64_t bl = smem_desc(smem_u32(Blo) + boff, 1024, 2);
#pragma unroll
            for (int mt = 0; mt < C::MT; ++mt) {
              const uint32_t aoff = (uint32_t)(mt * 128 * C::ROWB + ks * 32);
              const uint64_t ah = smem_desc(abase + aoff, 8 * C::ROWB, alayout);
              const uint64_t al = smem_desc(abase + C::AHALF + aoff, 8 * C::ROWB, alayout);
              const uint32_t dt = tmem + C::TM_Z + mt * NS;
              const int first = (c == 0 && ks == 0);
              mma_tf32(dt, ah, bh, idesc, first ? 0 : 1);
              mma_tf32(dt, ah, bl, idesc, 1);
              mma_tf32(dt, al, bh, idesc, 1);
            }
          }
          mma_commit(empty + st);   // the stage is free once these MMAs have read it
          ++gc;
        }
        if (!ok) break;
        mma_commit(zready);         // Z of this GEMM is complete
        ++gmm;
      }
      // wind down: copies still in flight complete before the CTA exits
      if (loaded > gc) tc_wait(full + (int)(gc & 1), (unsigned)((gc >> 1) & 1), 1 << 20, abort_flag, p.status);
      if (gc > 0) {   // the last MMAs have completed (their stage's commit)
        const long x = gc - 1;
        mbar_wait(empty + (int)(x & 1), (unsigned)((x >> 1) & 1), 1 << 20);
      }
    }
    __syncwarp();
  } else {
    // ============================================================== epilogue (128 threads)
    const int et = threadIdx.x - 32;                   // 0..255
    const int eg = et >> 7;                            // column group: chunks cc = eg, eg + 2, ...
    const int L = 32 * (warp & 3) + lane;              // TMEM lane = output row within a tile
    const uint32_t lane_addr = (uint32_t)(32 * (warp & 3)) << 16;
    const int ew = warp & 3;                           // epilogue warp index for the z partials
    long gmm = 0;
    const Cheb<float>* chp = reinterpret_cast<const Cheb<float>*>(p.cheb);

    // per-state set-up for step s: control, sub-interval parameters, activity
    auto setup = [&](int s) {
      if (et < NI) {
        const TcItem it = p.items[item0 + et];
        TcPar& q = par[et];
        int n = -1, j = 0;
        bool on = it.b >= 0;
        if (on) {
          if (p.mode == 0) {
            j = it.dir == 0 ? s : p.Nt - 1 - s;
            on = s < p.Nt;
            if (q.n < 0) q.n = it.dir == 0 ? 0 : p.N - 1;   // first sub-interval of the sweep
            n = q.n;
          } else {
            n = it.n;
            const int ns = p.jn[n + 1] - p.jn[n];
            on = s < ns;
            j = p.jn[n] + (s < ns ? s : ns - 1);
          }
        }
        if (n >= 0 && q.ln != n) {   // load the sub-interval's parameters
          const Cheb<float>& ch = chp[(long)it.b * p.N + n];
          const float sg = (p.mode == 0 && it.dir == 1) ? -1.f : 1.f;
          for (int k = 0; k < KMAX; ++k) {
            const float s_k = (k & 1) ? sg : 1.f;
            q.ch[k] = s_k * ch.cf[k];
            q.cl[k] = s_k * ch.cl[k];
          }
          q.ch[0] = ch.c0h; q.cl[0] = ch.c0l;           // a_0 - 1: the step is v + Delta
          q.ch[1] = sg * ch.a1h; q.cl[1] = sg * ch.a1l;
          split2<float>(ch.s2d, q.s2h, q.s2l);
          split2<float>(ch.cd * ch.s2d, q.cs2h, q.cs2l);
          q.K = ch.K;
          q.S = ch.S;
          q.cph = ch.cph;
          q.sph = ch.sph;
          q.ln = n;
        }
        q.u = on ? p.uf[(long)it.b * p.Nt + j] : 0.f;
        q.on = on ? 1 : 0;
        if (on) q.work += (unsigned long long)q.S;
      }
      epi_sync();
      if (et == 0) {
        int K = 2, S = 1;
        for (int i = 0; i < NI; ++i)
          if (par[i].on || (p.mode == 1 && p.items[item0 + i].b >= 0)) { K = max(K, par[i].K); S = max(S, par[i].S); }
        kt_st[0] = K;
        kt_st[1] = S;
      }
      epi_sync();
    };

    // initial states (FP64) -> FP32 hi + lo in the state scratch, and the B operand of the first GEMM
    for (int lt = 0; lt < C::LT; ++lt) {
      const int f = lt * 128 + L;
      for (int i = eg; i < NI; i += 2) {
        const TcItem it = p.items[item0 + i];
        double2 z = make_double2(0.0, 0.0);
        if (it.b >= 0) {
          const long off = (long)it.b * (p.N + 1) * D;
          if (p.mode == 0) {
            if (it.dir == 0) {
              z = p.psi_i[f];
              p.psin[off + f] = z;                                    // psi(t_0) = psi_i
            } else if (p.obj == 0) {
              z = p.psi_f[f];
              p.chin[off + (long)p.N * D + f] = z;                    // chi(T) = psi_f
            } else {
              z = p.chin[off + (long)p.N * D + f];                    // chi(T) = O psi(T), stored before
            }
          } else {
            z = (it.role == 0 ? p.psin : p.chin)[off + (long)it.n * D + f];
          }
        }
        const float re = (float)z.x, im = (float)z.y;
        vs[(size_t)(2 * i) * D + f] = re;
        vs[(size_t)(2 * i + 1) * D + f] = im;
        vs[(size_t)(NS + 2 * i) * D + f] = (float)(z.x - (double)re);
        vs[(size_t)(NS + 2 * i + 1) * D + f] = (float)(z.y - (double)im);
        const float rh = tf32_rn(re), ih = tf32_rn(im);
        *reinterpret_cast<float*>(Bhi + b_off<D>(2 * i, f)) = rh;
        *reinterpret_cast<float*>(Blo + b_off<D>(2 * i, f)) = tf32_rn(re - rh);
        *reinterpret_cast<float*>(Bhi + b_off<D>(2 * i + 1, f)) = ih;
        *reinterpret_cast<float*>(Blo + b_off<D>(2 * i + 1, f)) = tf32_rn(im - ih);
      }
    }
    if (et < NI) { par[et].n = -1; par[et].ln = -1; par[et].K = 0; par[et].work = 0; }
    epi_sync();

    // hand a GEMM to the MMA issuer (go = 1) or stop it (go = 0)
    auto release = [&](int go) {
      fence_proxy_async();   // this thread's B writes are visible to the tensor cores
      tmem_wait_st();
      tc_fence_before();
      epi_sync();
      if (et == 0) {
        *cmd = go;
        mbar_arrive(bready);
      }
    };
    auto await_z = [&]() -> bool {
      const bool ok = tc_wait(zready, (unsigned)(gmm & 1), p.max_spin, abort_flag, p.status);
      ++gmm;
      tc_fence_after();
      return ok;
    };

    const int last = p.mode == 1 ? p.nsteps : p.nsteps - 1;   // sub-interval sweeps: one more term-0 GEMM
    bool alive = true;
    for (int s = 0; s <= last && alive; ++s) {
      setup(s);
      const int Kt = kt_st[0], St = p.mode == 1 && s == p.nsteps ? 1 : kt_st[1];
      for (int sub = 0; sub < St && alive; ++sub) {
        for (int g = 0; g + 1 < Kt && alive; ++g) {
          release(1);
          if (!(alive = await_z())) break;
          const bool zterm = p.mode == 1 && g == 0 && sub == 0;   // overlaps <chi|H1 psi> from this Z
          const bool final_g = g + 2 == Kt || (p.mode == 1 && s == p.nsteps);
          for (int cc = eg; cc < NS / TC_CW; cc += 2) {
            float zloc[TC_CW / 4][2];   // the chunk's (psi, chi) pairs: columns 4q .. 4q+3
#pragma unroll
            for (int q2 = 0; q2 < TC_CW / 4; ++q2) { zloc[q2][0] = 0.f; zloc[q2][1] = 0.f; }
            for (int lt = 0; lt < C::LT; ++lt) {
              const int f = lt * 128 + L;
              float z0[TC_CW], z1[TC_CW], tp[TC_CW], ac[TC_CW];
              tmem_ld16(tmem + lane_addr + C::TM_Z + lt * NS + cc * TC_CW, z0);
              tmem_ld16(tmem + lane_addr + C::TM_Z + (C::LT + lt) * NS + cc * TC_CW, z1);
              if (g > 0) {
                tmem_ld16(tmem + lane_addr + C::TM_TP + lt * NS + cc * TC_CW, tp);
                tmem_ld16(tmem + lane_addr + C::TM_AC + lt * NS + cc * TC_CW, ac);
              }
              tmem_wait_ld();
              if (p.mode == 1 && s == p.nsteps) {   // terminal overlap only
#pragma unroll
                for (int q2 = 0; q2 < TC_CW / 4; ++q2) {
                  const int cb = cc * TC_CW + 4 * q2;
                  const float hr = z1[4 * q2], hi = z1[4 * q2 + 1];
                  const float xr = *reinterpret_cast<const float*>(Bhi + b_off<D>(cb + 2, f)) +
                                   *reinterpret_cast<const float*>(Blo + b_off<D>(cb + 2, f));
                  const float xi = *reinterpret_cast<const float*>(Bhi + b_off<D>(cb + 3, f)) +
                                   *reinterpret_cast<const float*>(Blo + b_off<D>(cb + 3, f));
                  zloc[q2][0] += xr * hr + xi * hi;
                  zloc[q2][1] += xr * hi - xi * hr;
                }
                continue;
              }
#pragma unroll
              for (int m = 0; m < TC_CW / 2; ++m) {   // state i = cc*CW/2 + m: columns 2m (re), 2m+1 (im)
                const int i = cc * (TC_CW / 2) + m;
                const TcPar& q = par[i];
                const int c0 = 2 * i;
                const uint32_t o0 = b_off<D>(c0, f), o1 = b_off<D>(c0 + 1, f);
                const float tr = *reinterpret_cast<const float*>(Bhi + o0) + *reinterpret_cast<const float*>(Blo + o0);
                const float ti = *reinterpret_cast<const float*>(Bhi + o1) + *reinterpret_cast<const float*>(Blo + o1);
                if (zterm && (m & 1)) {              // chi (odd state) against H1 psi (the even state)
                  const float hr = z1[2 * m - 2], hi = z1[2 * m - 1];
                  zloc[m >> 1][0] += tr * hr + ti * hi;
                  zloc[m >> 1][1] += tr * hi - ti * hr;
                }
                // Y T = 0.5 [s2 (Z0 + u Z1) - cs2 T]
                const float xr = fmaf(q.u, z1[2 * m], z0[2 * m]), xi = fmaf(q.u, z1[2 * m + 1], z0[2 * m + 1]);
                float yr = fmaf(q.s2h, xr, fmaf(q.s2l, xr, -fmaf(q.cs2h, tr, q.cs2l * tr)));
                float yi = fmaf(q.s2h, xi, fmaf(q.s2l, xi, -fmaf(q.cs2h, ti, q.cs2l * ti)));
                float nr, ni;
                if (g == 0) {
                  nr = 0.5f * yr;
                  ni = 0.5f * yi;
                  // the series sum starts at (a_0 - 1) T_0
                  ac[2 * m] = fmaf(q.ch[0], tr, q.cl[0] * tr);
                  ac[2 * m + 1] = fmaf(q.ch[0], ti, q.cl[0] * ti);
                } else {
                  nr = yr - tp[2 * m];
                  ni = yi - tp[2 * m + 1];
                }
                // + a_{g+1} (-i)^{g+1} T_{g+1} (the signs of (-i)^k and of the adjoint are folded into ch)
                const int k = g + 1;
                const float ck = q.ch[k], cl = q.cl[k];
                if (k & 1) {
                  ac[2 * m] = fmaf(ck, ni, fmaf(cl, ni, ac[2 * m]));
                  ac[2 * m + 1] = fmaf(-ck, nr, fmaf(-cl, nr, ac[2 * m + 1]));
                } else {
                  ac[2 * m] = fmaf(ck, nr, fmaf(cl, nr, ac[2 * m]));
                  ac[2 * m + 1] = fmaf(ck, ni, fmaf(cl, ni, ac[2 * m + 1]));
                }
                tp[2 * m] = tr;
                tp[2 * m + 1] = ti;
                if (!final_g) {   // T_{g+1} is the next GEMM's B operand
                  const float rh = tf32_rn(nr), ih = tf32_rn(ni);
                  *reinterpret_cast<float*>(Bhi + o0) = rh;
                  *reinterpret_cast<float*>(Blo + o0) = tf32_rn(nr - rh);
                  *reinterpret_cast<float*>(Bhi + o1) = ih;
                  *reinterpret_cast<float*>(Blo + o1) = tf32_rn(ni - ih);
                } else {          // end of the sub-step: v <- v + Delta (two-sum), B <- v
                  const bool adv = q.on && sub < q.S;
                  float* vh0 = vs + (size_t)c0 * D + f;
                  float* vl0 = vs + (size_t)(NS + c0) * D + f;
                  float vr = vh0[0], vi = vh0[D], lr = vl0[0], li = vl0[D];
                  if (adv) {
                    float t = ac[2 * m] + lr, sm2 = vr + t, bb = sm2 - vr;
                    lr = (vr - (sm2 - bb)) + (t - bb);
                    vr = sm2;
                    t = ac[2 * m + 1] + li; sm2 = vi + t; bb = sm2 - vi;
                    li = (vi - (sm2 - bb)) + (t - bb);
                    vi = sm2;
                    vh0[0] = vr; vh0[D] = vi; vl0[0] = lr; vl0[D] = li;
                  }
                  const float rh = tf32_rn(vr), ih = tf32_rn(vi);
                  *reinterpret_cast<float*>(Bhi + o0) = rh;
                  *reinterpret_cast<float*>(Blo + o0) = tf32_rn(vr - rh);
                  *reinterpret_cast<float*>(Bhi + o1) = ih;
                  *reinterpret_cast<float*>(Blo + o1) = tf32_rn(vi - ih);
                }
              }
              if (!final_g) {
                tmem_st16(tmem + lane_addr + C::TM_TP + lt * NS + cc * TC_CW, tp);
                tmem_st16(tmem + lane_addr + C::TM_AC + lt * NS + cc * TC_CW, ac);
              }
            }
            if (zterm || (p.mode == 1 && s == p.nsteps)) {   // the chunk's pair sums over this warp's rows
#pragma unroll
              for (int q2 = 0; q2 < TC_CW / 4; ++q2)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                  float v = zloc[q2][h];
                  for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                  if (lane == 0) zred[(ew * (NI / 2) + cc * (TC_CW / 4) + q2) * 2 + h] = v;
                }
            }
          }
          if (zterm || (p.mode == 1 && s == p.nsteps)) {   // sum the four warps' partials; one slot per pair
            epi_sync();
            if (et < NI / 2) {
              const TcItem it = p.items[item0 + 2 * et];
              if (it.b >= 0) {
                const int n = it.n, ns = p.jn[n + 1] - p.jn[n];
                if (s <= ns) {
                  float zr = 0.f, zi = 0.f;
                  for (int w4 = 0; w4 < 4; ++w4) { zr += zred[(w4 * (NI / 2) + et) * 2]; zi += zred[(w4 * (NI / 2) + et) * 2 + 1]; }
                  p.zs[(long)it.b * (p.Nt + p.N) + p.jn[n] + n + s] = make_float2(zr, zi);
                }
              }
            }
          }
          if (p.mode == 1 && s == p.nsteps) break;
        }
      }
      // global sweeps: the state at each partition point, with the segment phase applied in FP64
      if (p.mode == 0 && alive) {
        epi_sync();
        for (int i = eg; i < NI; i += 2) {
          const TcItem it = p.items[item0 + i];
          if (it.b < 0) continue;
          TcPar& q = par[i];
          const int j = it.dir == 0 ? s : p.Nt - 1 - s;
          const int n = q.n;
          const bool at = it.dir == 0 ? (j + 1 == p.jn[n + 1]) : (j == p.jn[n]);
          if (!at) continue;
          const long off = (long)it.b * (p.N + 1) * D;
          double2* dst = it.dir == 0 ? p.psin + off + (long)(n + 1) * D : p.chin + off + (long)n * D;
          for (int lt = 0; lt < C::LT; ++lt) {
            const int f = lt * 128 + L;
            float* vh0 = vs + (size_t)(2 * i) * D + f;
            float* vl0 = vs + (size_t)(NS + 2 * i) * D + f;
            double yr, yi;
            phase_rotate(q.cph, q.sph, it.dir == 1, (double)vh0[0] + (double)vl0[0], (double)vh0[D] + (double)vl0[D], yr, yi);
            dst[f] = make_double2(yr, yi);
            const float re = (float)yr, im = (float)yi;
            vh0[0] = re; vh0[D] = im;
            vl0[0] = (float)(yr - (double)re); vl0[D] = (float)(yi - (double)im);
            const float rh = tf32_rn(re), ih = tf32_rn(im);
            *reinterpret_cast<float*>(Bhi + b_off<D>(2 * i, f)) = rh;
            *reinterpret_cast<float*>(Blo + b_off<D>(2 * i, f)) = tf32_rn(re - rh);
            *reinterpret_cast<float*>(Bhi + b_off<D>(2 * i + 1, f)) = ih;
            *reinterpret_cast<float*>(Blo + b_off<D>(2 * i + 1, f)) = tf32_rn(im - ih);
          }
        }
        epi_sync();
        if (et < NI) {   // next sub-interval of the items that crossed a partition point
          const TcItem it = p.items[item0 + et];
          TcPar& q = par[et];
          if (it.b >= 0) {
            const int j = it.dir == 0 ? s : p.Nt - 1 - s;
            if (it.dir == 0 && j + 1 == p.jn[q.n + 1] && q.n + 1 < p.N) q.n += 1;
            else if (it.dir == 1 && j == p.jn[q.n] && q.n > 0) q.n -= 1;
          }
        }
      }
    }
    release(0);   // stop the MMA issuer
    if (et < NI && p.count && p.items[item0 + et].b >= 0) {
      const TcPar& q = par[et];
      atomicAdd(p.count + 0, q.work * (unsigned long long)(q.K - 1));
      atomicAdd(p.count + 1, q.work * (unsigned long long)q.K);
      atomicAdd(p.count + 2, q.work);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, 512);
}

// chi(T) = O psi(T) in FP64, one CTA per problem
__global__ void k_tc_chiT(const double* O, const double2* psin, double2* chin, int d, int N) {
  const int b = blockIdx.x;
  const double2* psT = psin + ((long)b * (N + 1) + N) * d;
  double2* chT = chin + ((long)b * (N + 1) + N) * d;
  for (int e = threadIdx.x; e < d; e += blockDim.x) {
    double sr = 0.0, si = 0.0;
    for (int f = 0; f < d; ++f) {
      const double o = O[(long)e * d + f];
      sr = fma(o, psT[f].x, sr);
      si = fma(o, psT[f].y, si);
    }
    chT[e] = make_double2(sr, si);
  }
}

typedef CUresult (*EncodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

template <int D>
cudaError_t launch_d(const TcMaps& m, const TcParams& p, cudaStream_t st) {
  using C = TcCfg<D>;
  const size_t smem = tc_smem_bytes(D);
  static_assert(sizeof(CUtensorMap) == 128, "tensor map size");
  cudaError_t e = cudaFuncSetAttribute(k_tc_sweep<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  CUtensorMap hi, lo;
  std::memcpy(&hi, m.hi, sizeof(hi));
  std::memcpy(&lo, m.lo, sizeof(lo));
  const int blocks = p.nitems / C::NI;
  k_tc_sweep<D><<<blocks, TC_THREADS, smem, st>>>(hi, lo, p);
  return cudaGetLastError();
}

}  // namespace

bool tc_supported(int d) { return d == 128 || d == 256; }
int tc_items_per_cta(int d) { return d == 128 ? TcCfg<128>::NI : TcCfg<256>::NI; }

size_t tc_smem_bytes(int d) {
  auto f = [](int BHALF, int STAGE, int NI) {
    return (size_t)1024 + 2 * BHALF + 2 * STAGE + NI * sizeof(TcPar) + 4 * NI * sizeof(float) + 8 * sizeof(uint64_t) + 64;
  };
  return d == 128 ? f(TcCfg<128>::BHALF, TcCfg<128>::STAGE, TcCfg<128>::NI)
                  : f(TcCfg<256>::BHALF, TcCfg<256>::STAGE, TcCfg<256>::NI);
}

cudaError_t tc_encode_maps(TcMaps* m, const float* hi, const float* lo, int d) {
  static EncodeTiled enc = nullptr;
  if (!enc) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || !fn || q != cudaDriverEntryPointSuccess) return e != cudaSuccess ? e : cudaErrorNotSupported;
    enc = reinterpret_cast<EncodeTiled>(fn);
  }
  const int kc = d == 128 ? TcCfg<128>::KC : TcCfg<256>::KC;
  const int boxr = 2 * d < 256 ? 2 * d : 256;
  const CUtensorMapSwizzle sw = kc * 4 == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B;
  cuuint64_t dims[2] = {(cuuint64_t)d, (cuuint64_t)(2 * d)};
  cuuint64_t strides[1] = {(cuuint64_t)d * sizeof(float)};
  cuuint32_t box[2] = {(cuuint32_t)kc, (cuuint32_t)boxr};
  cuuint32_t estr[2] = {1, 1};
  CUtensorMap th, tl;
  CUresult r = enc(&th, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(hi), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r == CUDA_SUCCESS)
    r = enc(&tl, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(lo), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  std::memcpy(m->hi, &th, sizeof(th));
  std::memcpy(m->lo, &tl, sizeof(tl));
  return cudaSuccess;
}

cudaError_t launch_tc_sweep(const TcMaps& m, const TcParams& p, cudaStream_t st) {
  if (p.d == 128) return launch_d<128>(m, p, st);
  if (p.d == 256) return launch_d<256>(m, p, st);
  return cudaErrorInvalidValue;
}

cudaError_t launch_tc_chiT(const double* O, double2* psin, double2* chin, int d, int N, int B, cudaStream_t st) {
  k_tc_chiT<<<B, 128, 0, st>>>(O, psin, chin, d, N);
  return cudaGetLastError();
}

}  // namespace ism

namespace ism {
namespace {

// Algorithm 1 step (c) after the stacked sub-interval sweep: one warp per (problem, n) forms the
// trapezoid gradient from the stored overlaps z_s = <chi_s|H1 psi_s> (two-trajectory form: no phase,
// scale 1/beta_n unless p.global), J_n from the FP64 boundary states, Err and the ascent step.
__global__ void __launch_bounds__(128) k_tc_zgrad(KParams p) {
  const long gid = (long)blockIdx.x * 4 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (gid >= (long)p.B * p.N) return;
  const int n = (int)(gid % p.N), b = (int)(gid / p.N);
  const int j0 = p.jn[n], ns = p.jn[n + 1] - j0;
  const double beta = p.beta[n];
  const long off = ((long)b * (p.N + 1) + n + 1) * p.d;
  double nrm = 0.0;
  for (int e = lane; e < p.d; e += 32) {
    const double2 x = p.chin[off + e], y = p.psin[off + e];
    const double dr = (x.x - y.x) / beta, di = (x.y - y.y) / beta;
    nrm += dr * dr + di * di;
  }
  nrm = g_sum<32>(nrm);
  const float2* zs = reinterpret_cast<const float2*>(p.zs) + (long)b * (p.Nt + p.N) + j0 + n;
  sub_grad_pass<32, false, false>(p, zs, b, n, gid, j0, ns, 1.0, 0.0, nrm, lane, 32, true);
}

}  // namespace

cudaError_t launch_tc_zgrad(const KParams& p, cudaStream_t st) {
  const long items = (long)p.B * p.N;
  k_tc_zgrad<<<(unsigned)((items + 3) / 4), 128, 0, st>>>(p);
  return cudaGetLastError();
}

}  // namespace ism
