// Tensor-core Legendre stages for FP32 plans with a lambda table
// (HPX_PLAN_TENSOR_CORES; Sec. III-D Eq. 14, Eq. 24-27).
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
// The synthesis is the same product the other way round:
//   D[p][n] = sum_l Lambda[l][p] At[n][l],
// At holding P_l a_lm split by the parity of l - m, so that the columns give
// E (even) and O (odd) and the rings get E + O (north) and E - O (south).
// Its lambda tiles come from a column copy of the table, [p][l] blocks of
// 128 pairs x 32 l, so that both operands are K-major as in the analysis.
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

#include <climits>
#include <vector>

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
// ---------------------------------------------------------------------------
// synthesis operands
// ---------------------------------------------------------------------------
// Coefficient operand At[m][j][n][32] for l = m + 32 j + (0..31): row n < 2 CP
// holds part n%2 of P_l mfac a_lm of channel n/2 where l - m is even (0
// elsewhere), row 2 CP + n the same for odd l - m; zero past lmax.  Only
// Re a_l0 enters (real maps).  One warp per (m, j).
template <int CP>
__global__ void __launch_bounds__(128)
k_pack_at(const float2* __restrict__ alm, const double* __restrict__ coef_p, const long long* __restrict__ achunk,
          float* __restrict__ at, int lmax, int mmax, long long nalm, int b0, int nb, double mfac) {
  constexpr int C2N = 2 * CP, NN = 2 * C2N;
  const int m = blockIdx.y, j = blockIdx.x * 4 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (m > mmax || j > (lmax - m) / 32) return;
  const int l = m + 32 * j + lane;
  float* out = at + (achunk[m] + j) * NN * 32 + lane;
  const bool in = l <= lmax;
  const bool odd = ((l - m) & 1) != 0;
  const long long base = alm_base(lmax, m);
  const double s = in ? coef_p[base + l] * (m > 0 ? mfac : 1.0) : 0.0;
#pragma unroll 4
  for (int c = 0; c < CP; ++c) {
    float2 a = make_float2(0.f, 0.f);
    if (in && c < nb) {
      a = alm[(long long)(b0 + c) * nalm + base + l];
      a = make_float2((float)(s * a.x), m == 0 ? 0.f : (float)(s * a.y));
    }
    const float2 e = odd ? make_float2(0.f, 0.f) : a, o = odd ? a : make_float2(0.f, 0.f);
    out[(2 * c) * 32] = e.x;
    out[(2 * c + 1) * 32] = e.y;
    out[(C2N + 2 * c) * 32] = o.x;
    out[(C2N + 2 * c + 1) * 32] = o.y;
  }
}

// Column lambda table for the synthesis: per (m, tile T of 128 ring pairs),
// from ls_T = the tile's first significant l (aligned down to m + 32 j) to
// lmax, blocks of 128 pairs x 32 l, element [p][l] = the recurrence value of
// chain (m, 128 T + p) in the same float as the row table (zero before the
// chain's start, past lmax and for pairs past npair).
__global__ void k_stab_tiles(const int* __restrict__ lc_tab, int lmax, int npair, int nptile, int* lstart,
                             long long* nblk) {
  const int T = blockIdx.x * blockDim.x + threadIdx.x, m = blockIdx.y;
  if (T >= nptile) return;
  int ls = lmax + 1;
  for (int j = 0; j < 128; ++j) {
    const int p = T * 128 + j;
    if (p < npair) ls = min(ls, lc_tab[(long long)m * npair + p]);
  }
  if (ls <= lmax) ls = m + ((ls - m) / 32) * 32;
  lstart[(long long)m * nptile + T] = ls;
  nblk[(long long)m * nptile + T] = ls <= lmax ? (lmax - ls) / 32 + 1 : 0;
}

__global__ void k_stab_fill(const RingInfo* __restrict__ rings, const double* __restrict__ coef_c,
                            const int* __restrict__ lc_tab, const double* __restrict__ mu0_tab,
                            const double* __restrict__ mu1_tab, const int* __restrict__ lstart,
                            const long long* __restrict__ off, int lmax, int npair, int nptile, float* tab) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x, m = blockIdx.y;
  const int T = p >> 7;
  if (T >= nptile) return;
  const long long mT = (long long)m * nptile + T;
  const int ls = lstart[mT];
  if (ls > lmax) return;
  const int lend = ls + ((lmax - ls) / 32 + 1) * 32;  // end of the last block
  float* out = tab + off[mT] + (p & 127) * 32;
  double z = 0.0, s0 = 0.0, s1 = 0.0;
  int lc = INT_MAX;
  if (p < npair) {
    const long long ci = (long long)m * npair + p;
    z = rings[p].z;
    lc = lc_tab[ci];
    s0 = mu0_tab[ci];
    s1 = mu1_tab[ci];
  }
  const long long base = alm_base(lmax, m);
  double mu1 = 0.0, mu2 = 0.0;
  for (int l4 = ls; l4 < lend; l4 += 4) {
    float v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int l = l4 + u;
      float f = 0.f;
      if (l <= lmax && p < npair) {  // the row table's recurrence, operation for operation
        double mu = fma(coef_c[base + l] * z, mu1, -mu2);
        if (l == lc) {
          mu = s1;
          mu1 = s0;
        }
        mu2 = mu1;
        mu1 = mu;
        f = to_real<float>(mu);
      }
      v[u] = f;
    }
    const int r = l4 - ls;
    *reinterpret_cast<float4*>(out + (long long)(r >> 5) * 4096 + (r & 31)) = make_float4(v[0], v[1], v[2], v[3]);
  }
}

// ---------------------------------------------------------------------------
// the tile kernels
// ---------------------------------------------------------------------------
template <int NN>
struct TcShape {
  static constexpr int kA = kTcTile * 128;   // lambda tile bytes: 128 rows x 32 floats
  static constexpr int kG = NN * 128;        // B tile bytes (Gt or At)
  static constexpr int kStage = kA + 2 * kG; // one stage: lambda tile, B tile, its remainder right after it
  static constexpr int kLo = kA;             // lambda remainder buffer (two, alternating by K block)
  static constexpr int kNStage = (200 * 1024 - 2 * kLo) / kStage < 8 ? (200 * 1024 - 2 * kLo) / kStage : 8;
  static constexpr int kTmemCols = 4 * NN;   // two block accumulators of 2 NN columns
  static constexpr size_t kSmem =
      (size_t)kNStage * kStage + 2 * kLo + 1024 /* base alignment */ + 2048 /* barriers, lists */;
  static_assert(kNStage >= 2 && kTmemCols <= 512, "shape");
};

constexpr int kTcThreads = 192;  // warps 0-3 split and drain, warp 4 copies, warp 5 issues products

struct TcArgs {
  const long long* off;    // analysis: row table offsets [m][group]; synthesis: column table [m][p tile]
  const int* lstart;       // first l stored, same indexing
  int ngroup;              // groups (analysis) or p tiles (synthesis) per m
  const long long* achunk; // synthesis: first At chunk of each m
  const double* coef_p;    // analysis: P_l
  float* out;              // analysis: alm [b][nalm] complex; synthesis: F [b][nring][mmax+1] complex
  int lmax, mmax, npair, nring;
  long long nalm;
  int b0, nb;
  double mfac;
  int* status;
};

// One CTA: a 128-row tile of one m, all channels of the launch.
//   analysis (SYN false): rows are l = l0 .. l0+127, K runs over the 32-pair
//     groups whose table rows reach the tile, B = Gt: D[l][n] = sum_p L G;
//   synthesis (SYN true): rows are ring pairs p = 128 T .. 128 T + 127, K runs
//     over 32-l chunks from the tile's first significant l, A = the column
//     table's blocks, B = At: D[p][n] = sum_l L^T At.
// Per K block k, with L the lambda tile (128 x 32) and B (NN x 32) in shared
// memory:
//   split: lo(L) and lo(B) are formed (hi is the hardware's TF32 truncation
//          of the tile as loaded; lo = x - trunc(x), rounded to TF32);
//          lo(B) sits right after B, so [B; lo B] is one N = 2 NN operand;
//   products (4 steps of K = 8): D[:, 0:2NN] += L [B; lo B]^T and
//          D[:, 0:NN] += lo(L) B^T, i.e. 8 instructions per block;
//   drain: D[r][j] + D[r][NN + j] is added into FP32 registers (round to
//          nearest): the NN/2 columns of the row's parity (analysis) or all
//          NN (synthesis).
// The tensor cores add each instruction's products into the accumulator
// with truncation, so each block is accumulated alone, in one of two TMEM
// buffers (2 NN columns each), while the other is drained.
//
// Roles run decoupled, linked by mbarriers: warp 4 keeps up to kNStage
// blocks of copies in flight, warp 5 issues a block's products once it is
// split and its accumulator is free, warps 0-3 split block k and then drain
// block k-1.  After an expired wait a role stops working (the split/drain
// warps keep looping without work, so their warp-collective tcgen05.ld stays
// convergent), waits for what it started, and the CTA records the timeout.
template <int NN, bool SYN>
__global__ void __launch_bounds__(kTcThreads, 1)
k_legendre_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const TcArgs a) {
  using S = TcShape<NN>;
  constexpr int NS = S::kNStage, C2N = NN / 2;
  constexpr int NSUM = SYN ? NN : C2N;
  static_assert(NN % 32 == 0 && NN <= 128, "N tile");
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int m = blockIdx.y;
  const int l0 = m + kTcTile * blockIdx.x;  // analysis tile
  if (!SYN && l0 > a.lmax) return;          // whole CTA, before any shared state

  extern __shared__ unsigned char smem_raw[];
  unsigned char* tiles = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* lobuf = tiles + (size_t)NS * S::kStage;
  uint64_t* full = reinterpret_cast<uint64_t*>(lobuf + 2 * S::kLo);
  uint64_t* conv = full + NS;   // stage split (128 arrivals)
  uint64_t* empty = conv + NS;  // stage's products done
  uint64_t* accf = empty + NS;  // [2] block accumulator complete
  uint64_t* acce = accf + 2;    // [2] block accumulator drained (128 arrivals)
  uint64_t* done = acce + 2;    // all products done
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  int* wcount = reinterpret_cast<int*>(tmem_slot + 2);  // [4]
  int* rowA = wcount + 4;   // analysis: [128] TMA row of the lambda tile of active group k
  int* rowB = rowA + 128;   // analysis: [128] TMA row of its Gt tile
  auto sL = [&](int s) { return tiles + (size_t)s * S::kStage; };
  auto sB = [&](int s) { return tiles + (size_t)s * S::kStage + S::kA; };
  auto sBlo = [&](int s) { return tiles + (size_t)s * S::kStage + S::kA + S::kG; };
  auto sLlo = [&](int b) { return lobuf + (size_t)b * S::kLo; };

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(S::kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  // K blocks.  Analysis: groups whose rows reach this tile (group starts lie
  // on the tile grid m + 128 j, so a group covers the whole tile or starts
  // after it), with their copy coordinates, compacted in group order.
  // Synthesis: every 32-l chunk from the tile's first stored l.
  bool act = false;
  int ra = 0, rb = 0;
  unsigned bal = 0;
  if (!SYN && warp < 4) {
    if (t < a.ngroup) {
      const long long mg = (long long)m * a.ngroup + t;
      const int ls = a.lstart[mg];
      act = ls <= l0;
      ra = (int)(a.off[mg] / 32) + (l0 - ls);
      rb = (int)(mg * NN);
    }
    bal = __ballot_sync(0xffffffffu, act);
    if (lane == 0) wcount[warp] = __popc(bal);
  }
  int na = 0, ra0 = 0, rb0 = 0;  // synthesis: block count, first rows
  if (SYN) {
    const long long mT = (long long)m * a.ngroup + blockIdx.x;
    const int ls = a.lstart[mT];
    if (ls <= a.lmax) {
      na = (a.lmax - ls) / 32 + 1;
      ra0 = (int)(a.off[mT] / 32);
      rb0 = (int)((a.achunk[m] + (ls - m) / 32) * NN);
    }
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
  if (!SYN) {
    if (act) {
      int off = 0;
      for (int w = 0; w < warp; ++w) off += wcount[w];
      const int k = off + __popc(bal & ((1u << lane) - 1u));
      rowA[k] = ra;
      rowB[k] = rb;
    }
    na = wcount[0] + wcount[1] + wcount[2] + wcount[3];
  }
  const uint32_t tmem = *tmem_slot;
  __syncthreads();

  if (warp == 4) {
    // ---- copies: block k into stage k % NS once block k - NS's products are done
    int issued = 0;
    if (lane == 0) {
      for (int k = 0; k < na; ++k) {
        const int s = k % NS;
        if (k >= NS && !wait_phase(&empty[s], (uint32_t)(k / NS - 1) & 1u, abort_flag, true)) break;
        mbar_expect_tx(&full[s], S::kA + S::kG);
        tma_load_2d(sL(s), &tmA, 0, SYN ? ra0 + k * 128 : rowA[k], &full[s]);
        tma_load_2d(sB(s), &tmB, 0, SYN ? rb0 + k * NN : rowB[k], &full[s]);
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
        const uint32_t aL = smem_u32(sL(s)), aLlo = smem_u32(sLlo(b)), aB = smem_u32(sB(s));
#pragma unroll
        for (int j = 0; j < 4; ++j) {  // K = 8 floats (32 bytes) per instruction
          const uint32_t off = 32u * j;
          umma_tf32(d, sdesc_sw128(aL + off), sdesc_sw128(aB + off), id2, j > 0 ? 1u : 0u);
          umma_tf32(d, sdesc_sw128(aLlo + off), sdesc_sw128(aB + off), id1, 1u);
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
    // ---- split and drain (thread t owns TMEM lane t = row t of the tile)
    const int l = l0 + t;
    const bool odd = ((l - m) & 1) != 0;
    const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
    float sum[NSUM];
#pragma unroll
    for (int j = 0; j < NSUM; ++j) sum[j] = 0.f;
    auto drain = [&](int buf) {  // warp-collective
      const uint32_t c0 = trow + (uint32_t)(buf * 2 * NN);
      if constexpr (SYN) {
#pragma unroll
        for (int q = 0; q < NN / 16; ++q) {
          uint32_t v1[16], v2[16];
          tmem_ld16(c0 + (uint32_t)(q * 16), v1);
          tmem_ld16(c0 + (uint32_t)(NN + q * 16), v2);
          tmem_wait_ld();
#pragma unroll
          for (int j = 0; j < 16; ++j) sum[q * 16 + j] += __uint_as_float(v1[j]) + __uint_as_float(v2[j]);
        }
      } else {
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
      }
    };
    bool alive = true;
    for (int k = 0; k < na; ++k) {
      const int s = k % NS, b = k & 1;
      if (alive) alive = wait_phase(&full[s], (uint32_t)(k / NS) & 1u, abort_flag, true);
      if (alive) {
        // elementwise, so the swizzle does not matter; consecutive threads
        // take consecutive 16-byte words.  Remainder buffer b was last read
        // by block k-2's products, complete since this thread drained that
        // block in the previous iteration.
        const float4* x = reinterpret_cast<const float4*>(sL(s));
        float4* xlo = reinterpret_cast<float4*>(sLlo(b));
#pragma unroll
        for (int j = 0; j < S::kA / 2048; ++j) xlo[j * 128 + t] = tf32_rem4(x[j * 128 + t]);
        const float4* y = reinterpret_cast<const float4*>(sB(s));
        float4* ylo = reinterpret_cast<float4*>(sBlo(s));
#pragma unroll
        for (int j = 0; j < S::kG / 2048; ++j) ylo[j * 128 + t] = tf32_rem4(y[j * 128 + t]);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(&conv[s]);
      }
      if (k >= 1) {  // drain block k-1 while block k's products run
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
    if (na > 0) {  // the last block
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
    if (*abort_flag == 0) {
      if constexpr (SYN) {
        // north ring p: E + O; its mirror (none for the equator): E - O
        const int p = blockIdx.x * 128 + t;
        if (p < a.npair) {
          const int ys = p == a.npair - 1 ? -1 : a.nring - 1 - p;
          float2* F = reinterpret_cast<float2*>(a.out);
          const long long mstride = a.mmax + 1;
#pragma unroll
          for (int c = 0; c < C2N / 2; ++c) {
            if (c < a.nb) {
              const float er = sum[2 * c], ei = sum[2 * c + 1], orr = sum[C2N + 2 * c], oi = sum[C2N + 2 * c + 1];
              const long long fb = (long long)(a.b0 + c) * a.nring;
              F[(fb + p) * mstride + m] = make_float2(er + orr, ei + oi);
              if (ys >= 0) F[(fb + ys) * mstride + m] = make_float2(er - orr, ei - oi);
            }
          }
        }
      } else if (l <= a.lmax) {
        const long long base = alm_base(a.lmax, m);
        const double scale = a.coef_p[base + l] * (m > 0 ? a.mfac : 1.0);
        float2* out = reinterpret_cast<float2*>(a.out) + (long long)a.b0 * a.nalm + base + l;
#pragma unroll
        for (int c = 0; c < C2N / 2; ++c)
          if (c < a.nb)
            out[(long long)c * a.nalm] =
                make_float2((float)(scale * sum[2 * c]), (float)(scale * sum[2 * c + 1]));
      }
    }
    if (*abort_flag != 0 && t == 0) atomicExch(a.status, (int)HPX_ERR_TIMEOUT);
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

TcArgs tc_args(const hpx_plan_s* p, bool syn, float* out, int b0, int nb, double mfac) {
  TcArgs a;
  a.off = syn ? p->d_stab_off : p->d_tab_off;
  a.lstart = syn ? p->d_stab_lstart : p->d_tab_lstart;
  a.ngroup = syn ? p->nptile : p->ngroup;
  a.achunk = p->d_achunk;
  a.coef_p = p->d_coef_p;
  a.out = out;
  a.lmax = p->lmax;
  a.mmax = p->mmax;
  a.npair = p->npair;
  a.nring = p->nring;
  a.nalm = p->nalm;
  a.b0 = b0;
  a.nb = nb;
  a.mfac = mfac;
  a.status = p->d_status;
  return a;
}

template <int CP>
cudaError_t launch_pack_cp(const hpx_plan_s* p, int b0, int nb, bool use_w, cudaStream_t s) {
  k_pack_gt<CP><<<dim3((p->ngroup + 3) / 4, p->mmax + 1), 128, 0, s>>>(
      (const float2*)p->d_spec, (const float2*)p->d_etab, p->d_ring, (float*)p->d_gt, p->npair, p->nring, p->ngroup,
      p->nspec, b0, nb, use_w ? 1 : 0);
  return cudaGetLastError();
}

template <int CP>
cudaError_t launch_pack_at_cp(const hpx_plan_s* p, const float* alm, int b0, int nb, double mfac, cudaStream_t s) {
  const int nchunk0 = p->lmax / 32 + 1;  // chunks of m = 0, the most
  k_pack_at<CP><<<dim3((nchunk0 + 3) / 4, p->mmax + 1), 128, 0, s>>>(
      (const float2*)alm, p->d_coef_p, p->d_achunk, (float*)p->d_at, p->lmax, p->mmax, p->nalm, b0, nb, mfac);
  return cudaGetLastError();
}

template <int CP, bool SYN>
cudaError_t launch_tile_cp(const hpx_plan_s* p, float* out, int b0, int nb, double mfac, cudaStream_t s) {
  constexpr int NN = 4 * CP;
  cudaError_t e = allow_max_smem(k_legendre_tc<NN, SYN>);
  if (e != cudaSuccess) return e;
  const CUtensorMap* tmA = reinterpret_cast<const CUtensorMap*>(SYN ? p->tm_stab : p->tm_tab);
  const CUtensorMap* tmB = reinterpret_cast<const CUtensorMap*>(SYN ? p->tm_at : p->tm_gt);
  const dim3 grid(SYN ? p->nptile : (p->lmax + kTcTile) / kTcTile, p->mmax + 1);
  k_legendre_tc<NN, SYN><<<grid, kTcThreads, TcShape<NN>::kSmem, s>>>(*tmA, *tmB,
                                                                       tc_args(p, SYN, out, b0, nb, mfac));
  return cudaGetLastError();
}

}  // namespace

int tc_columns(int nbatch) {
  int cp = 8;
  while (cp < nbatch && cp < 32) cp *= 2;
  return 4 * cp;
}

int tc_channels_per_launch(const hpx_plan_s* p) { return p->tc_nn / 4; }

size_t tc_extra_bytes_estimate(int nside, int lmax, int mmax, int nbatch) {
  const size_t npair = 2 * (size_t)nside, ngroup = (npair + 31) / 32, nptile = (npair + 127) / 128;
  const size_t nn = (size_t)tc_columns(nbatch);
  size_t chunks = 0;
  for (int m = 0; m <= mmax; ++m) chunks += (size_t)((lmax - m) / 32 + 1);
  return sizeof(float) * (size_t)(mmax + 1) * ngroup * nn * 32     // Gt
         + sizeof(float) * chunks * nn * 32                         // At
         + sizeof(float) * chunks * nptile * 128 * 32               // column table (upper bound)
         + (sizeof(int) + sizeof(long long)) * (size_t)(mmax + 1) * nptile + sizeof(long long) * (mmax + 2);
}

cudaError_t build_tc(hpx_plan_s* p, cudaStream_t s) {
  const int nn = tc_columns(p->nbatch);
  // analysis operand
  size_t elems = (size_t)(p->mmax + 1) * p->ngroup * nn * 32;
  cudaError_t e = cudaMalloc(&p->d_gt, elems * sizeof(float));
  if (e != cudaSuccess) return e;
  p->bytes += elems * sizeof(float);
  // synthesis operand: chunk offsets of each m, then At
  std::vector<long long> ach(p->mmax + 2);
  ach[0] = 0;
  for (int m = 0; m <= p->mmax; ++m) ach[m + 1] = ach[m] + (p->lmax - m) / 32 + 1;
  e = cudaMalloc((void**)&p->d_achunk, sizeof(long long) * (p->mmax + 2));
  if (e != cudaSuccess) return e;
  p->bytes += sizeof(long long) * (p->mmax + 2);
  e = cudaMemcpy(p->d_achunk, ach.data(), sizeof(long long) * (p->mmax + 2), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return e;
  elems = (size_t)ach[p->mmax + 1] * nn * 32;
  e = cudaMalloc(&p->d_at, elems * sizeof(float));
  if (e != cudaSuccess) return e;
  p->bytes += elems * sizeof(float);
  // column table
  p->nptile = (p->npair + 127) / 128;
  const long long nent = (long long)(p->mmax + 1) * p->nptile;
  e = cudaMalloc((void**)&p->d_stab_lstart, sizeof(int) * nent);
  if (e != cudaSuccess) return e;
  p->bytes += sizeof(int) * nent;
  e = cudaMalloc((void**)&p->d_stab_off, sizeof(long long) * nent);
  if (e != cudaSuccess) return e;
  p->bytes += sizeof(long long) * nent;
  k_stab_tiles<<<dim3((p->nptile + 127) / 128, p->mmax + 1), 128, 0, s>>>(p->d_lc, p->lmax, p->npair, p->nptile,
                                                                           p->d_stab_lstart, p->d_stab_off);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e;
  std::vector<long long> off(nent);
  e = cudaMemcpy(off.data(), p->d_stab_off, sizeof(long long) * nent, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return e;
  long long acc = 0;
  for (long long i = 0; i < nent; ++i) {
    const long long nb = off[i];
    off[i] = acc;
    acc += nb * 128 * 32;
  }
  p->stab_elems = acc;
  e = cudaMemcpy(p->d_stab_off, off.data(), sizeof(long long) * nent, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return e;
  e = cudaMalloc(&p->d_stab, sizeof(float) * (acc > 0 ? acc : 32));
  if (e != cudaSuccess) return e;
  p->bytes += sizeof(float) * (acc > 0 ? acc : 32);
  k_stab_fill<<<dim3(p->nptile, p->mmax + 1), 128, 0, s>>>(p->d_ring, p->d_coef_c, p->d_lc, p->d_mu0, p->d_mu1,
                                                           p->d_stab_lstart, p->d_stab_off, p->lmax, p->npair,
                                                           p->nptile, static_cast<float*>(p->d_stab));
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const unsigned long long at_rows = (unsigned long long)ach[p->mmax + 1] * nn;
  if (!encode_rows32(p->tm_tab, p->d_tab, (unsigned long long)(p->tab_elems / 32), kTcTile) ||
      !encode_rows32(p->tm_gt, p->d_gt, (unsigned long long)(p->mmax + 1) * p->ngroup * nn, nn) ||
      !encode_rows32(p->tm_stab, p->d_stab, (unsigned long long)(acc > 0 ? acc / 32 : 1), 128) ||
      !encode_rows32(p->tm_at, p->d_at, at_rows, nn)) {
    set_error("cuTensorMapEncodeTiled failed or is unavailable");
    return cudaErrorInvalidValue;
  }
  p->tc_nn = nn;
  return cudaSuccess;
}

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
    case 32: return launch_tile_cp<8, false>(p, alm, b0, nb, mfac, s);
    case 64: return launch_tile_cp<16, false>(p, alm, b0, nb, mfac, s);
    case 128: return launch_tile_cp<32, false>(p, alm, b0, nb, mfac, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_pack_at_tc(const hpx_plan_s* p, const float* alm, int b0, int nb, double mfac, cudaStream_t s) {
  switch (p->tc_nn) {
    case 32: return launch_pack_at_cp<8>(p, alm, b0, nb, mfac, s);
    case 64: return launch_pack_at_cp<16>(p, alm, b0, nb, mfac, s);
    case 128: return launch_pack_at_cp<32>(p, alm, b0, nb, mfac, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_synthesis_tc(const hpx_plan_s* p, int b0, int nb, cudaStream_t s) {
  float* F = static_cast<float*>(p->d_F);
  switch (p->tc_nn) {
    case 32: return launch_tile_cp<8, true>(p, F, b0, nb, 1.0, s);
    case 64: return launch_tile_cp<16, true>(p, F, b0, nb, 1.0, s);
    case 128: return launch_tile_cp<32, true>(p, F, b0, nb, 1.0, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace hpx
