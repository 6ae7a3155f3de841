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
// each float (10 mantissa bits).  Each operand is split as x = hi + lo with
// hi = x rounded to the nearest TF32 value, so |lo| <= 2^-11 |x| and lo is
// exact in FP32; lo is itself rounded to TF32 (error <= 2^-22 |x|).  Then
//   D = hi(L) hi(G) + hi(L) lo(G) + lo(L) hi(G)
// ("3xTF32", the split-operand scheme of Markidis et al. 2018 and Ootomo &
// Yokota 2022) has a relative error of at most about 3 x 2^-22 per product
// (the two rounded remainders and the dropped lo*lo term), accumulated in
// FP32 in tensor memory.  The split is done in shared memory on each landed
// tile: hi overwrites the tile, lo goes to a second one.
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

constexpr int kStagesMax = 4;
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
// Splits a tile element in place: hi = tf32_rn(x) stays, lo = tf32_rn(x - hi)
// (x - hi is exact in FP32) goes to the remainder tile.
__device__ __forceinline__ void split4(float4& x, float4& lo) {
  const float4 h = make_float4(tf32_rn(x.x), tf32_rn(x.y), tf32_rn(x.z), tf32_rn(x.w));
  lo = make_float4(tf32_rn(x.x - h.x), tf32_rn(x.y - h.y), tf32_rn(x.z - h.z), tf32_rn(x.w - h.w));
  x = h;
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
  static constexpr int kA = kTcTile * 128;        // lambda tile bytes: 128 rows x 32 floats
  static constexpr int kG = NN * 128;             // Gt tile bytes
  static constexpr int kStage = 2 * kA + 2 * kG;  // L, lo L, G, lo G
  static constexpr int kNStage = (kStagesMax * kStage <= 200 * 1024) ? kStagesMax : (200 * 1024) / kStage;
  static constexpr int kTmemCols = 2 * NN;        // two group accumulators
  static constexpr size_t kSmem = (size_t)kNStage * kStage + 1024 /* base alignment */ + 1024 /* barriers, list */;
};

// One CTA: rows l0 .. l0+127 of one m, all channels of the launch.
//
// Accumulation: the tensor cores add each instruction's products into the
// accumulator with truncation, so one accumulator over all K would collect
// an error growing with the number of ring pairs.  Each 32-pair group is
// therefore accumulated alone (12 instructions) in one of two TMEM buffers
// and added, with round-to-nearest FP32 adds, into per-thread register sums
// while the next group's products run in the other buffer.
//
// Roles: thread 0 issues the TMA copies, thread 32 the MMAs, all 128
// threads split the landed tiles and drain the accumulators (thread t owns
// TMEM lane t = row l0 + t).  No thread leaves the group loop early: after an
// expired wait a thread only stops doing work, so the warp-collective
// tcgen05.ld stays convergent.
template <int NN>
__global__ void __launch_bounds__(128, 1)
k_analysis_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmG,
              const long long* __restrict__ tab_off, const int* __restrict__ lstart, int ngroup,
              const double* __restrict__ coef_p, float* __restrict__ alm, int lmax, long long nalm, int b0, int nb,
              double mfac, int* __restrict__ status) {
  using S = TcShape<NN>;
  constexpr int NS = S::kNStage, C2N = NN / 2;
  static_assert(NN % 32 == 0 && NN <= 256, "N tile");
  const int t = threadIdx.x, warp = t >> 5;
  const int m = blockIdx.y;
  const int l0 = m + kTcTile * blockIdx.x;
  if (l0 > lmax) return;  // whole CTA, before any shared state

  extern __shared__ unsigned char smem_raw[];
  unsigned char* tiles = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(tiles + (size_t)NS * S::kStage);
  uint64_t* conv = full + NS;   // tile split (128 arrivals)
  uint64_t* empty = conv + NS;  // stage's products done
  uint64_t* accf = empty + NS;  // [2] group accumulator complete
  uint64_t* acce = accf + 2;    // [2] group accumulator drained (128 arrivals)
  uint64_t* done = acce + 2;    // all products done
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  int* nact = reinterpret_cast<int*>(tmem_slot + 2);
  int* glist = nact + 1;  // groups reaching this tile, in order (ngroup <= 128)
  auto sL = [&](int s) { return tiles + (size_t)s * S::kStage; };
  auto sLlo = [&](int s) { return tiles + (size_t)s * S::kStage + S::kA; };
  auto sG = [&](int s) { return tiles + (size_t)s * S::kStage + 2 * S::kA; };
  auto sGlo = [&](int s) { return tiles + (size_t)s * S::kStage + 2 * S::kA + S::kG; };

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(S::kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
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
    // group starts lie on the tile grid m + 128 j, so a group either covers
    // the whole tile or starts after it
    int n = 0;
    for (int g = 0; g < ngroup; ++g)
      if (lstart[(long long)m * ngroup + g] <= l0) glist[n++] = g;
    *nact = n;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const int na = *nact;

  auto issue_loads = [&](int k) {  // thread 0
    const int s = k % NS, g = glist[k];
    const long long mg = (long long)m * ngroup + g;
    const int row = (int)(tab_off[mg] / 32) + (l0 - lstart[mg]);
    mbar_expect_tx(&full[s], S::kA + S::kG);
    tma_load_2d(sL(s), &tmA, 0, row, &full[s]);
    tma_load_2d(sG(s), &tmG, 0, (int)(mg * NN), &full[s]);
  };
  int issued = 0;
  if (t == 0)
    for (; issued < na && issued < NS; ++issued) issue_loads(issued);

  // row l = l0 + t keeps the columns of its parity: S (n < C2N) for even
  // l - m, A for odd
  const int l = l0 + t;
  const bool odd = ((l - m) & 1) != 0;
  const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
  float sum[C2N];
#pragma unroll
  for (int j = 0; j < C2N; ++j) sum[j] = 0.f;
  auto drain = [&](int buf) {  // warp-collective
#pragma unroll
    for (int q = 0; q < C2N / 16; ++q) {
      uint32_t rs[16], ra[16];
      tmem_ld16(trow + (uint32_t)(buf * NN + q * 16), rs);
      tmem_ld16(trow + (uint32_t)(buf * NN + C2N + q * 16), ra);
      tmem_wait_ld();
#pragma unroll
      for (int j = 0; j < 16; ++j) sum[q * 16 + j] += __uint_as_float(odd ? ra[j] : rs[j]);
    }
  };

  // instruction descriptor: D f32, A and B tf32, both K-major, N = NN, M = 128
  const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(NN >> 3) << 17) | ((128u >> 4) << 24);
  bool alive = true, mma_issued = false;
  for (int k = 0; k < na; ++k) {
    const int s = k % NS;
    const uint32_t ph = (uint32_t)(k / NS) & 1u;
    if (alive) alive = wait_phase(&full[s], ph, abort_flag, true);
    if (alive) {  // split 32 lambda floats and NN/4 Gt floats per thread
      float4* a = reinterpret_cast<float4*>(sL(s)) + t * 8;
      float4* alo = reinterpret_cast<float4*>(sLlo(s)) + t * 8;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        float4 x = a[j], lo;
        split4(x, lo);
        a[j] = x;
        alo[j] = lo;
      }
      float4* gg = reinterpret_cast<float4*>(sG(s)) + t * (NN / 16);
      float4* glo = reinterpret_cast<float4*>(sGlo(s)) + t * (NN / 16);
#pragma unroll
      for (int j = 0; j < NN / 16; ++j) {
        float4 x = gg[j], lo;
        split4(x, lo);
        gg[j] = x;
        glo[j] = lo;
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(&conv[s]);
    }
    if (t == 32 && alive) {
      alive = wait_phase(&conv[s], ph, abort_flag, true);
      if (alive && k >= 2) alive = wait_phase(&acce[k & 1], (uint32_t)((k - 2) >> 1) & 1u, abort_flag, true);
      if (alive) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t d = tmem + (uint32_t)((k & 1) * NN);
        const uint32_t aL = smem_u32(sL(s)), aLlo = smem_u32(sLlo(s)), aG = smem_u32(sG(s)),
                       aGlo = smem_u32(sGlo(s));
#pragma unroll
        for (int j = 0; j < 4; ++j) {  // K = 8 floats (32 bytes) per instruction
          const uint32_t off = 32u * j;
          umma_tf32(d, sdesc_sw128(aL + off), sdesc_sw128(aG + off), idesc, j > 0 ? 1u : 0u);
          umma_tf32(d, sdesc_sw128(aL + off), sdesc_sw128(aGlo + off), idesc, 1u);
          umma_tf32(d, sdesc_sw128(aLlo + off), sdesc_sw128(aG + off), idesc, 1u);
        }
        umma_commit(&empty[s]);
        umma_commit(&accf[k & 1]);
        mma_issued = true;
      }
    }
    if (t == 0 && alive && k >= 1 && issued < na) {  // refill the stage group k-1 used once its products are done
      alive = wait_phase(&empty[(k - 1) % NS], (uint32_t)((k - 1) / NS) & 1u, abort_flag, true);
      if (alive) issue_loads(issued++);
    }
    __syncwarp();
    if (k >= 1) {  // drain group k-1 while group k's products run
      bool ok = alive && wait_phase(&accf[(k - 1) & 1], (uint32_t)((k - 1) >> 1) & 1u, abort_flag, true);
      ok = __all_sync(0xffffffffu, ok);
      if (ok) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        drain((k - 1) & 1);
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        mbar_arrive(&acce[(k - 1) & 1]);
      } else {
        alive = false;
      }
    }
  }
  // every product and copy this CTA started completes before the last
  // drain, or before the tensor memory is released after an abort
  if (t == 32 && mma_issued) {
    umma_commit(done);
    wait_phase(done, 0, abort_flag, false);
  }
  if (t == 0)
    for (int k = issued > NS ? issued - NS : 0; k < issued; ++k)
      wait_phase(&full[k % NS], (uint32_t)(k / NS) & 1u, abort_flag, false);
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (*abort_flag == 0) {
    if (na > 0) drain((na - 1) & 1);
    if (l <= lmax) {
      const long long base = alm_base(lmax, m);
      const double scale = coef_p[base + l] * (m > 0 ? mfac : 1.0);
      float2* out = reinterpret_cast<float2*>(alm) + (long long)b0 * nalm + base + l;
#pragma unroll
      for (int c = 0; c < C2N / 2; ++c)
        if (c < nb) out[(long long)c * nalm] = make_float2((float)(scale * sum[2 * c]), (float)(scale * sum[2 * c + 1]));
    }
  } else if (t == 0) {
    atomicExch(status, (int)HPX_ERR_TIMEOUT);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(S::kTmemCols));
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
cudaError_t launch_cp(const hpx_plan_s* p, float* alm, bool use_w, double mfac, cudaStream_t s, int* nlaunch) {
  constexpr int NN = 4 * CP;
  using Sh = TcShape<NN>;
  cudaError_t e = allow_max_smem(k_analysis_tc<NN>);
  if (e != cudaSuccess) return e;
  const CUtensorMap* tmA = reinterpret_cast<const CUtensorMap*>(p->tm_tab);
  const CUtensorMap* tmG = reinterpret_cast<const CUtensorMap*>(p->tm_gt);
  const dim3 tiles((p->lmax + kTcTile) / kTcTile, p->mmax + 1);
  for (int b0 = 0; b0 < p->nbatch; b0 += CP) {
    const int nb = (p->nbatch - b0) < CP ? (p->nbatch - b0) : CP;
    k_pack_gt<CP><<<dim3((p->ngroup + 3) / 4, p->mmax + 1), 128, 0, s>>>(
        (const float2*)p->d_spec, (const float2*)p->d_etab, p->d_ring, (float*)p->d_gt, p->npair, p->nring,
        p->ngroup, p->nspec, b0, nb, use_w ? 1 : 0);
    k_analysis_tc<NN><<<tiles, 128, Sh::kSmem, s>>>(*tmA, *tmG, p->d_tab_off, p->d_tab_lstart, p->ngroup,
                                                    p->d_coef_p, alm, p->lmax, p->nalm, b0, nb, mfac, p->d_status);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    *nlaunch += 2;
  }
  return cudaSuccess;
}

}  // namespace

int tc_columns(int nbatch) {
  int cp = 8;
  while (cp < nbatch && cp < 64) cp *= 2;
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

cudaError_t launch_analysis_tc(const hpx_plan_s* p, float* alm, bool use_w, double mfac, cudaStream_t s,
                               int* nlaunch) {
  switch (p->tc_nn) {
    case 32: return launch_cp<8>(p, alm, use_w, mfac, s, nlaunch);
    case 64: return launch_cp<16>(p, alm, use_w, mfac, s, nlaunch);
    case 128: return launch_cp<32>(p, alm, use_w, mfac, s, nlaunch);
    case 256: return launch_cp<64>(p, alm, use_w, mfac, s, nlaunch);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace hpx
