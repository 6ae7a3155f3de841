// Tensor-core Legendre analysis for FP32 plans with a lambda table
// (HPX_PLAN_TENSOR_CORES; Sec. III-D Eq. 14, Eq. 26-27).
//
// For one m the analysis is a matrix product over ring pairs p:
//   D[l][n] = sum_p Lambda[l][p] Gt[n][p],
// with n over the real components of S_m (used by even l - m) and A_m (odd
// l - m) of every channel: N = 2 parities x 2 parts x channels.  Both parities
// are formed for every row and the epilogue keeps the row's own: the table
// stream, not the tensor pipe, bounds the kernel.  One CTA owns 128
// consecutive l of one m (M = 128); its K loop runs over the 32-pair groups
// whose table rows reach the tile.  A lambda tile (128 rows x 32 floats, one
// 128-byte swizzle atom along K) and a Gt tile (N rows x 32 floats) arrive by
// TMA in a shared-memory ring of stages; tcgen05.mma accumulates in tensor
// memory and tcgen05.ld brings the tile back for the epilogue (times P_l).
//
// FP32 accuracy from TF32 products: the tensor cores read the top 19 bits of
// each float (10 mantissa bits), i.e. hi(x) = x truncated to TF32.  With
// lo(x) = x - hi(x) (exact in FP32, |lo| < 2^-10 |x|) rounded to TF32,
//   D = hi(L) hi(G) + hi(L) lo(G) + lo(L) hi(G)
// ("3xTF32", the split-operand scheme of Markidis et al. 2018 and Ootomo &
// Yokota 2022) drops the lo*lo term and the rounding of the remainders:
// about 2^-20 relative per product at worst, 2^-22 typically.  The
// remainders are formed in shared memory from each landed tile.
//
// Every mbarrier wait is bounded in time.  When one expires the CTA stops
// issuing work, waits (again bounded) for the copies and products it has in
// flight, records HPX_ERR_TIMEOUT in the plan's status word, frees its tensor
// memory and returns; its output rows are then left unwritten.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "hpx_internal.cuh"

namespace hpx {
namespace {

constexpr unsigned long long kWaitNs = 1000000000ull;  // 1 s per wait

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for the phase of `bar` with the given parity.  Gives up (false) when
// another thread of the CTA has raised the abort flag (if watch_abort) or
// after kWaitNs, raising the flag itself.
__device__ bool wait_phase(uint64_t* bar, uint32_t parity, volatile int* abort_flag, bool watch_abort) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (unsigned i = 1; i < (1u << 31); ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 63u) == 0) {
      if (watch_abort && *abort_flag) return false;
      if (global_ns() - t0 > kWaitNs) break;
    }
  }
  *abort_flag = 1;
  return false;
}
__device__ __forceinline__ void tma_load_2d(void* dst, const void* map, int c0, int c1, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"((uint64_t)map), "r"(c0), "r"(c1), "r"(smem_u32(bar))
      : "memory");
}
// Shared-memory matrix descriptor of a K-major operand in the 128-byte
// swizzle: rows of 128 bytes, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
__device__ __forceinline__ void umma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
// 16 consecutive accumulator columns of this warp's 32 TMEM lanes (complete
// after tmem_wait_ld).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
// x rounded to the nearest TF32 value (ties away from zero): the 13 low
// mantissa bits rounded into the upper 19.  Finite inputs of table and
// spectrum magnitude only (no overflow to infinity can occur there).
__device__ __forceinline__ float tf32_rn(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}
// The part of x the tensor cores drop (they read the TF32 truncation of x),
// exact in FP32, itself rounded to TF32.
__device__ __forceinline__ float tf32_rem(float x) {
  return tf32_rn(x - __uint_as_float(__float_as_uint(x) & 0xFFFFE000u));
}
__device__ __forceinline__ float4 tf32_rem4(float4 x) {
  return make_float4(tf32_rem(x.x), tf32_rem(x.y), tf32_rem(x.z), tf32_rem(x.w));
}

// ---------------------------------------------------------------------------
// operand pack: Gt[m][g][n][32] from the ring spectra
// ---------------------------------------------------------------------------
// For pair p (north ring p, south ring nring-1-p; the equator ring pairs with
// nothing) G(y) = W_y X_y[m mod N] exp(-i m phi_0) as in the CUDA-core
// analysis; row n < 2 CP holds part n%2 of S = G(north) + G(south) for channel
// n/2, row 2 CP + n that of A = G(north) - G(south).  One warp per group.
template <int CP>
__global__ void __launch_bounds__(128)
k_pack_gt(const float2* __restrict__ spec, const float2* __restrict__ etab, const RingInfo* __restrict__ rings,
          float* __restrict__ gt, int npair, int nring, int ngroup, long long nspec, int b0, int nb, int use_w) {
  constexpr int C2N = 2 * CP, NN = 2 * C2N;
  const int g = blockIdx.x * 4 + (threadIdx.x >> 5), m = blockIdx.y, lane = threadIdx.x & 31;
  if (g >= ngroup) return;
  const int p = g * 32 + lane;
  float* out = gt + ((long long)m * ngroup + g) * NN * 32 + lane;
  const bool active = p < npair;
  const bool has_south = active && p != npair - 1;
  int k = 0, N = 2;
  float2 en = make_float2(0.f, 0.f), es = en;
  long long on = 0, os = 0;
  float wn = 1.f, ws = 1.f;
  if (active) {
    const RingInfo Rn = rings[p];
    N = Rn.nphi;
    k = m % N;
    en = etab[Rn.etab + ((long long)Rn.sigma * m) % (2LL * N)];
    on = Rn.specoff;
    if (use_w) wn = (float)Rn.w;
    if (has_south) {  // mirror ring: same length, same table
      const RingInfo Rs = rings[nring - 1 - p];
      es = etab[Rs.etab + ((long long)Rs.sigma * m) % (2LL * N)];
      os = Rs.specoff;
      if (use_w) ws = (float)Rs.w;
    }
  }
  const bool conj = k > (N >> 1);
  const int kk = conj ? N - k : k;
#pragma unroll 4
  for (int c = 0; c < CP; ++c) {
    float2 gn = make_float2(0.f, 0.f), gs = gn;
    if (active && c < nb) {
      const float2* X = spec + (long long)(b0 + c) * nspec;
      float2 x = X[on + kk];
      if (conj) x = cconj(x);
      gn = cscale(cmul(x, en), wn);
      if (has_south) {
        x = X[os + kk];
        if (conj) x = cconj(x);
        gs = cscale(cmul(x, es), ws);
      }
    }
    out[(2 * c) * 32] = gn.x + gs.x;
    out[(2 * c + 1) * 32] = gn.y + gs.y;
    out[(C2N + 2 * c) * 32] = gn.x - gs.x;
    out[(C2N + 2 * c + 1) * 32] = gn.y - gs.y;
  }
}

// ---------------------------------------------------------------------------
// the tile kernel
// ---------------------------------------------------------------------------
template <int NN>
struct TcShape {
  static constexpr int kA = kTcTile * 128;   // lambda tile bytes: 128 rows x 32 floats
  static constexpr int kG = NN * 128;        // Gt tile bytes
  static constexpr int kStage = kA + 2 * kG; // one stage: lambda tile, Gt tile, its remainder right after it
  static constexpr int kLo = kA;             // lambda remainder buffer (two, alternating by group)
  static constexpr int kNStage = (200 * 1024 - 2 * kLo) / kStage < 8 ? (200 * 1024 - 2 * kLo) / kStage : 8;
  static constexpr int kTmemCols = 4 * NN;   // two group accumulators of 2 NN columns
  static constexpr size_t kSmem =
      (size_t)kNStage * kStage + 2 * kLo + 1024 /* base alignment */ + 2048 /* barriers, lists */;
  static_assert(kNStage >= 2 && kTmemCols <= 512, "shape");
};

constexpr int kTcThreads = 192;  // warps 0-3 split and drain, warp 4 copies, warp 5 issues products

// One CTA: rows l0 .. l0+127 of one m, all channels of the launch.
//
// Per 32-pair group k, with L the lambda tile (128 x 32) and G the operand
// tile (NN x 32) in shared memory:
//   split: lo(L) and lo(G) are formed (hi is the hardware's TF32 truncation
//          of the tile as loaded; lo = x - trunc(x), rounded to TF32);
//          lo(G) sits right after G, so [G; lo G] is one N = 2 NN operand;
//   products (4 steps of K = 8): D[:, 0:2NN] += L [G; lo G]^T and
//          D[:, 0:NN] += lo(L) G^T, i.e. 8 instructions per group;
//   drain: row l keeps D[l][j] + D[l][NN + j] for the NN/2 columns j of its
//          parity and adds them into FP32 registers (round to nearest).
// The tensor cores add each instruction's products into the accumulator
// with truncation, so each group is accumulated alone, in one of two TMEM
// buffers (2 NN columns each), while the other is drained.
//
// Roles run decoupled, linked by mbarriers: warp 4 keeps up to kNStage
// groups of copies in flight, warp 5 issues a group's products once it is
// split and its accumulator is free, warps 0-3 split group k and then drain
// group k-1.  After an expired wait a role stops working (the split/drain
// warps keep looping without work, so their warp-collective tcgen05.ld stays
// convergent), waits for what it started, and the CTA records the timeout.
template <int NN>
__global__ void __launch_bounds__(kTcThreads, 1)
k_analysis_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmG,
              const long long* __restrict__ tab_off, const int* __restrict__ lstart, int ngroup,
              const double* __restrict__ coef_p, float* __restrict__ alm, int lmax, long long nalm, int b0, int nb,
              double mfac, int* __restrict__ status) {
  using S = TcShape<NN>;
  constexpr int NS = S::kNStage, C2N = NN / 2;
  static_assert(NN % 32 == 0 && NN <= 128, "N tile");
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int m = blockIdx.y;
  const int l0 = m + kTcTile * blockIdx.x;
  if (l0 > lmax) return;  // whole CTA, before any shared state

  extern __shared__ unsigned char smem_raw[];
  unsigned char* tiles = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* lobuf = tiles + (size_t)NS * S::kStage;
  uint64_t* full = reinterpret_cast<uint64_t*>(lobuf + 2 * S::kLo);
  uint64_t* conv = full + NS;   // stage split (128 arrivals)
  uint64_t* empty = conv + NS;  // stage's products done
  uint64_t* accf = empty + NS;  // [2] group accumulator complete
  uint64_t* acce = accf + 2;    // [2] group accumulator drained (128 arrivals)
  uint64_t* done = acce + 2;    // all products done
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  int* wcount = reinterpret_cast<int*>(tmem_slot + 2);  // [4]
  int* rowA = wcount + 4;   // [128] TMA row of the lambda tile of active group k
  int* rowG = rowA + 128;   // [128] TMA row of its Gt tile
  auto sL = [&](int s) { return tiles + (size_t)s * S::kStage; };
  auto sG = [&](int s) { return tiles + (size_t)s * S::kStage + S::kA; };
  auto sGlo = [&](int s) { return tiles + (size_t)s * S::kStage + S::kA + S::kG; };
  auto sLlo = [&](int b) { return lobuf + (size_t)b * S::kLo; };

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(S::kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  // groups whose rows reach this tile (group starts lie on the tile grid
  // m + 128 j, so a group covers the whole tile or starts after it), with
  // their copy coordinates, compacted in group order
  bool act = false;
  int ra = 0, rg = 0;
  unsigned bal = 0;
  if (warp < 4) {
    if (t < ngroup) {
      const long long mg = (long long)m * ngroup + t;
      const int ls = lstart[mg];
      act = ls <= l0;
      ra = (int)(tab_off[mg] / 32) + (l0 - ls);
      rg = (int)(mg * NN);
    }
    bal = __ballot_sync(0xffffffffu, act);
    if (lane == 0) wcount[warp] = __popc(bal);
  }
  if (t == 32) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&conv[s], 128);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accf[b], 1);
      mbar_init(&acce[b], 128);
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (act) {
    int off = 0;
    for (int w = 0; w < warp; ++w) off += wcount[w];
    const int k = off + __popc(bal & ((1u << lane) - 1u));
    rowA[k] = ra;
    rowG[k] = rg;
  }
  const int na = wcount[0] + wcount[1] + wcount[2] + wcount[3];
  const uint32_t tmem = *tmem_slot;
  __syncthreads();

  if (warp == 4) {
    // ---- copies: group k into stage k % NS once group k - NS's products are done
    int issued = 0;
    if (lane == 0) {
      for (int k = 0; k < na; ++k) {
        const int s = k % NS;
        if (k >= NS && !wait_phase(&empty[s], (uint32_t)(k / NS - 1) & 1u, abort_flag, true)) break;
        mbar_expect_tx(&full[s], S::kA + S::kG);
        tma_load_2d(sL(s), &tmA, 0, rowA[k], &full[s]);
        tma_load_2d(sG(s), &tmG, 0, rowG[k], &full[s]);
        issued = k + 1;
      }
      // whatever was started completes before the CTA moves on
      for (int k = issued > NS ? issued - NS : 0; k < issued; ++k)
        wait_phase(&full[k % NS], (uint32_t)(k / NS) & 1u, abort_flag, false);
    }
  } else if (warp == 5) {
    // ---- products
    if (lane == 0) {
      // instruction descriptors: D f32, A and B tf32, both K-major, M = 128
      const uint32_t id2 = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(2 * NN >> 3) << 17) | ((128u >> 4) << 24);
      const uint32_t id1 = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(NN >> 3) << 17) | ((128u >> 4) << 24);
      bool issued_any = false;
      for (int k = 0; k < na; ++k) {
        const int s = k % NS, b = k & 1;
        if (!wait_phase(&conv[s], (uint32_t)(k / NS) & 1u, abort_flag, true)) break;
        if (k >= 2 && !wait_phase(&acce[b], (uint32_t)((k - 2) >> 1) & 1u, abort_flag, true)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t d = tmem + (uint32_t)(b * 2 * NN);
        const uint32_t aL = smem_u32(sL(s)), aLlo = smem_u32(sLlo(b)), aG = smem_u32(sG(s));
#pragma unroll
        for (int j = 0; j < 4; ++j) {  // K = 8 floats (32 bytes) per instruction
          const uint32_t off = 32u * j;
          umma_tf32(d, sdesc_sw128(aL + off), sdesc_sw128(aG + off), id2, j > 0 ? 1u : 0u);
          umma_tf32(d, sdesc_sw128(aLlo + off), sdesc_sw128(aG + off), id1, 1u);
        }
        umma_commit(&empty[s]);
        umma_commit(&accf[b]);
        issued_any = true;
      }
      if (issued_any) {
        umma_commit(done);
        wait_phase(done, 0, abort_flag, false);
      }
    }
  } else {
    // ---- split and drain (thread t owns TMEM lane t = row l0 + t)
    const int l = l0 + t;
    const bool odd = ((l - m) & 1) != 0;
    const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
    float sum[C2N];
#pragma unroll
    for (int j = 0; j < C2N; ++j) sum[j] = 0.f;
    auto drain = [&](int buf) {  // warp-collective
      const uint32_t c0 = trow + (uint32_t)(buf * 2 * NN);
#pragma unroll
      for (int q = 0; q < C2N / 16; ++q) {
        uint32_t s1[16], s2[16], a1[16], a2[16];
        tmem_ld16(c0 + (uint32_t)(q * 16), s1);
        tmem_ld16(c0 + (uint32_t)(NN + q * 16), s2);
        tmem_ld16(c0 + (uint32_t)(C2N + q * 16), a1);
        tmem_ld16(c0 + (uint32_t)(NN + C2N + q * 16), a2);
        tmem_wait_ld();
#pragma unroll
        for (int j = 0; j < 16; ++j)
          sum[q * 16 + j] += odd ? __uint_as_float(a1[j]) + __uint_as_float(a2[j])
                                 : __uint_as_float(s1[j]) + __uint_as_float(s2[j]);
      }
    };
    bool alive = true;
    for (int k = 0; k < na; ++k) {
      const int s = k % NS, b = k & 1;
      if (alive) alive = wait_phase(&full[s], (uint32_t)(k / NS) & 1u, abort_flag, true);
      if (alive) {
        // elementwise, so the swizzle does not matter; consecutive threads
        // take consecutive 16-byte words.  Remainder buffer b was last read
        // by group k-2's products, complete since this thread drained that
        // group in the previous iteration.
        const float4* a = reinterpret_cast<const float4*>(sL(s));
        float4* alo = reinterpret_cast<float4*>(sLlo(b));
#pragma unroll
        for (int j = 0; j < S::kA / 2048; ++j) alo[j * 128 + t] = tf32_rem4(a[j * 128 + t]);
        const float4* gg = reinterpret_cast<const float4*>(sG(s));
        float4* glo = reinterpret_cast<float4*>(sGlo(s));
#pragma unroll
        for (int j = 0; j < S::kG / 2048; ++j) glo[j * 128 + t] = tf32_rem4(gg[j * 128 + t]);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(&conv[s]);
      }
      if (k >= 1) {  // drain group k-1 while group k's products run
        bool ok = alive && wait_phase(&accf[b ^ 1], (uint32_t)((k - 1) >> 1) & 1u, abort_flag, true);
        ok = __all_sync(0xffffffffu, ok);
        if (ok) {
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          drain(b ^ 1);
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          mbar_arrive(&acce[b ^ 1]);
        } else {
          alive = false;
        }
      }
    }
    if (na > 0) {  // the last group
      bool ok = alive && wait_phase(&accf[(na - 1) & 1], (uint32_t)((na - 1) >> 1) & 1u, abort_flag, true);
      ok = __all_sync(0xffffffffu, ok);
      if (ok) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        drain((na - 1) & 1);
      }
    }
    __syncwarp();
    // the CTA-wide sync below orders these writes after every role finished;
    // results are written only if no wait expired anywhere in the CTA
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (*abort_flag == 0 && l <= lmax) {
      const long long base = alm_base(lmax, m);
      const double scale = coef_p[base + l] * (m > 0 ? mfac : 1.0);
      float2* out = reinterpret_cast<float2*>(alm) + (long long)b0 * nalm + base + l;
#pragma unroll
      for (int c = 0; c < C2N / 2; ++c)
        if (c < nb)
          out[(long long)c * nalm] = make_float2((float)(scale * sum[2 * c]), (float)(scale * sum[2 * c + 1]));
    }
    if (*abort_flag != 0 && t == 0) atomicExch(status, (int)HPX_ERR_TIMEOUT);
    __syncthreads();
    if (warp == 0)
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(S::kTmemCols));
    return;
  }
  // warps 4 and 5: meet the split/drain warps at their two CTA-wide syncs
  __syncwarp();
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  __syncthreads();
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)f;
  }
  return fn;
}

// A row-major float matrix of `rows` rows x 32 columns, read as tiles of
// box_rows x 32 in the 128-byte swizzle; rows past the end read as zero.
bool encode_rows32(void* out, const void* base, unsigned long long rows, unsigned box_rows) {
  auto enc = tensor_map_encoder();
  if (!enc) return false;
  cuuint64_t dims[2] = {32, (cuuint64_t)rows};
  cuuint64_t strides[1] = {32 * sizeof(float)};
  cuuint32_t box[2] = {32, box_rows}, es[2] = {1, 1};
  return enc(reinterpret_cast<CUtensorMap*>(out), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims,
             strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int CP>
cudaError_t launch_pack_cp(const hpx_plan_s* p, int b0, int nb, bool use_w, cudaStream_t s) {
  k_pack_gt<CP><<<dim3((p->ngroup + 3) / 4, p->mmax + 1), 128, 0, s>>>(
      (const float2*)p->d_spec, (const float2*)p->d_etab, p->d_ring, (float*)p->d_gt, p->npair, p->nring, p->ngroup,
      p->nspec, b0, nb, use_w ? 1 : 0);
  return cudaGetLastError();
}

template <int CP>
cudaError_t launch_tile_cp(const hpx_plan_s* p, float* alm, int b0, int nb, double mfac, cudaStream_t s) {
  constexpr int NN = 4 * CP;
  cudaError_t e = allow_max_smem(k_analysis_tc<NN>);
  if (e != cudaSuccess) return e;
  const CUtensorMap* tmA = reinterpret_cast<const CUtensorMap*>(p->tm_tab);
  const CUtensorMap* tmG = reinterpret_cast<const CUtensorMap*>(p->tm_gt);
  const dim3 tiles((p->lmax + kTcTile) / kTcTile, p->mmax + 1);
  k_analysis_tc<NN><<<tiles, kTcThreads, TcShape<NN>::kSmem, s>>>(*tmA, *tmG, p->d_tab_off, p->d_tab_lstart, p->ngroup,
                                                          p->d_coef_p, alm, p->lmax, p->nalm, b0, nb, mfac,
                                                          p->d_status);
  return cudaGetLastError();
}

}  // namespace

int tc_columns(int nbatch) {
  int cp = 8;
  while (cp < nbatch && cp < 32) cp *= 2;
  return 4 * cp;
}

cudaError_t build_tc_analysis(hpx_plan_s* p) {
  const int nn = tc_columns(p->nbatch);
  const size_t elems = (size_t)(p->mmax + 1) * p->ngroup * nn * 32;
  cudaError_t e = cudaMalloc(&p->d_gt, elems * sizeof(float));
  if (e != cudaSuccess) return e;
  p->bytes += elems * sizeof(float);
  if (!encode_rows32(p->tm_tab, p->d_tab, (unsigned long long)(p->tab_elems / 32), kTcTile) ||
      !encode_rows32(p->tm_gt, p->d_gt, (unsigned long long)(p->mmax + 1) * p->ngroup * nn, nn)) {
    set_error("cuTensorMapEncodeTiled failed or is unavailable");
    return cudaErrorInvalidValue;
  }
  p->tc_nn = nn;
  return cudaSuccess;
}

int tc_channels_per_launch(const hpx_plan_s* p) { return p->tc_nn / 4; }

cudaError_t launch_pack_tc(const hpx_plan_s* p, int b0, int nb, bool use_w, cudaStream_t s) {
  switch (p->tc_nn) {
    case 32: return launch_pack_cp<8>(p, b0, nb, use_w, s);
    case 64: return launch_pack_cp<16>(p, b0, nb, use_w, s);
    case 128: return launch_pack_cp<32>(p, b0, nb, use_w, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_tile_tc(const hpx_plan_s* p, float* alm, int b0, int nb, double mfac, cudaStream_t s) {
  switch (p->tc_nn) {
    case 32: return launch_tile_cp<8>(p, alm, b0, nb, mfac, s);
    case 64: return launch_tile_cp<16>(p, alm, b0, nb, mfac, s);
    case 128: return launch_tile_cp<32>(p, alm, b0, nb, mfac, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace hpx
