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
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <climits>
#include <vector>

#include "hpx_internal.cuh"

namespace hpx {
namespace {

constexpr unsigned long long kWaitNs = 1000000000ull;  // 1 s per wait
// 16-bit lambda tables hold 2^9 lambda (|lambda_lm| <= sqrt((2l+1)/4pi) < 64
// for l < 25000, so 2^9 |lambda| < 2^15 stays in FP16 range), which keeps
// the FP16 remainder parts of small values out of the subnormal range; the
// epilogues multiply by 2^-9.
constexpr double kLamScale = 512.0;

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
__device__ __forceinline__ void umma_f16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
// A operand in tensor memory (lane = row, one 32-bit column per K element)
__device__ __forceinline__ void umma_tf32_ta(uint32_t d, uint32_t a_tmem, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}" ::"r"(d),
      "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc));
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
// 32 consecutive columns of this warp's 32 TMEM lanes, complete on return.
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,"
      "%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
      "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]), "r"(v[16]), "r"(v[17]), "r"(v[18]),
      "r"(v[19]), "r"(v[20]), "r"(v[21]), "r"(v[22]), "r"(v[23]), "r"(v[24]), "r"(v[25]), "r"(v[26]), "r"(v[27]),
      "r"(v[28]), "r"(v[29]), "r"(v[30]), "r"(v[31])
      : "memory");
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}
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
// operand element types
// ---------------------------------------------------------------------------
// float: FP32 tables and operands; the products are 3xTF32 with the
//   remainders made in shared memory (mode 0).
// __nv_bfloat16 / __half: 16-bit tables and operands (kind::f16 products,
//   FP32 accumulation); the hi part, and for the x3 modes the lo part
//   lo = x - hi rounded again, are stored (modes 1 and 2).
// A row of any operand tile is 128 bytes: 32 floats or 64 16-bit values.
template <typename E> struct Elt;
template <> struct Elt<float> {
  static constexpr int kw = 32;
  static __device__ __forceinline__ float from_float(float v) { return v; }
  static __device__ __forceinline__ float to_float(float v) { return v; }
};
template <> struct Elt<__nv_bfloat16> {
  static constexpr int kw = 64;
  static __device__ __forceinline__ __nv_bfloat16 from_float(float v) { return __float2bfloat16_rn(v); }
  static __device__ __forceinline__ float to_float(__nv_bfloat16 v) { return __bfloat162float(v); }
};
template <> struct Elt<__half> {
  static constexpr int kw = 64;
  static __device__ __forceinline__ __half from_float(float v) { return __float2half_rn(v); }
  static __device__ __forceinline__ float to_float(__half v) { return __half2float(v); }
};

// Operand value v (already scaled) into row n of a tile column: hi at row n,
// and for x3 the remainder at row NN + n.
template <typename E>
__device__ __forceinline__ void put(E* col, int n, int NN, float v, bool x3) {
  constexpr int KW = Elt<E>::kw;
  const E h = Elt<E>::from_float(v);
  col[(long long)n * KW] = h;
  if (x3) col[(long long)(NN + n) * KW] = Elt<E>::from_float(v - Elt<E>::to_float(h));
}

// Power of two s with s * bound <= 2^14, from the channel's recorded largest
// component |x| (bit pattern of a non-negative float) times sfac, so that
// FP16 operands stay in range; 1 without a record (FP32 operands) or for an
// all-zero channel.
__device__ __forceinline__ float chan_scale(const unsigned* bmax, int b, float sfac) {
  if (!bmax) return 1.f;
  const float amax = __uint_as_float(bmax[b]) * sfac;
  if (!(amax > 0.f) || !(amax < 3.0e38f)) return 1.f;
  int e;
  frexpf(amax, &e);  // amax < 2^e
  return ldexpf(1.f, min(14 - e, 126));  // 2^126 at most, so that the scale and its inverse are normal
}

// Largest |component| of each channel b0 .. b0+nb-1 of x ([b][stride]
// complex values, n per channel), as float bits, into bmax[b] (atomic max;
// zeroed first).
__global__ void k_absmax(const float2* __restrict__ x, long long n, long long stride, int b0, unsigned* bmax) {
  const int b = b0 + blockIdx.y;
  const float2* xb = x + (long long)b * stride;
  float v = 0.f;
  const long long step = (long long)gridDim.x * blockDim.x;
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i + 3 * step < n; i += 4 * step) {  // four loads in flight
    const float2 q0 = xb[i], q1 = xb[i + step], q2 = xb[i + 2 * step], q3 = xb[i + 3 * step];
    v = fmaxf(v, fmaxf(fmaxf(fabsf(q0.x), fabsf(q0.y)), fmaxf(fabsf(q1.x), fabsf(q1.y))));
    v = fmaxf(v, fmaxf(fmaxf(fabsf(q2.x), fabsf(q2.y)), fmaxf(fabsf(q3.x), fabsf(q3.y))));
  }
  for (; i < n; i += step) {
    const float2 q = xb[i];
    v = fmaxf(v, fmaxf(fabsf(q.x), fabsf(q.y)));
  }
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) atomicMax(bmax + b, __float_as_uint(v));
}

// ---------------------------------------------------------------------------
// analysis operand: Gt[m][g][rows][KW] from the ring spectra
// ---------------------------------------------------------------------------
// For pair p (north ring p, south ring nring-1-p; the equator ring pairs with
// nothing) G(y) = W_y X_y[m mod N] exp(-i m phi_0) as in the CUDA-core
// analysis; row n < 2 CP holds part n%2 of S = G(north) + G(south) for channel
// n/2, row 2 CP + n that of A = G(north) - G(south), times the channel's
// scale; for x3 rows NN .. 2 NN - 1 hold the remainders.
//
// One CTA: group g (KW pairs) x kPackM consecutive m x kPackC channels.  The
// spectra are read along m (kPackM consecutive bins of one ring and channel
// are contiguous), the values go to shared memory in the operand's row
// layout, and each m's rows leave as contiguous 128-byte lines.  A thread
// takes one (m, pair) at a time -- ring data, bin and phases once -- and
// all the CTA's channels of it.
constexpr int kPackM = 8, kPackC = 8;

__host__ __device__ constexpr int pack_rows(bool x3) { return (x3 ? 8 : 4) * kPackC; }  // shared rows per m
__host__ __device__ constexpr int pack_slab(int rows) { return rows * 128 + 16; }  // bytes; 16 against bank conflicts

template <typename E>
__global__ void __launch_bounds__(256)
k_pack_gt(const float2* __restrict__ spec, const float2* __restrict__ etab, const RingInfo* __restrict__ rings,
          E* __restrict__ gt, int npair, int nring, int ngroup, long long nspec, int mmax, int NN, int b0, int nb,
          int use_w, int x3, const unsigned* __restrict__ bmax, float sfac) {
  constexpr int KW = Elt<E>::kw;
  // dynamic shared memory only (the launch may raise its limit to the
  // device maximum): kPackM slabs, then the channel scales
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int g = blockIdx.x, m0 = blockIdx.y * kPackM, c0 = blockIdx.z * kPackC;
  const int C2N = NN / 2, rb = x3 ? 2 * NN : NN;
  const int rows = pack_rows(x3 != 0), slab = pack_slab(rows);
  float* csc = reinterpret_cast<float*>(smem_raw + kPackM * slab);
  if (threadIdx.x < kPackC) {
    const int c = c0 + threadIdx.x;
    csc[threadIdx.x] = c < nb ? chan_scale(bmax, b0 + c, sfac) : 0.f;
  }
  __syncthreads();
  const int nch = min(kPackC, nb - c0);  // channels with data; the rest are zero rows
  for (int i = threadIdx.x; i < kPackM * KW; i += blockDim.x) {
    const int ml = i % kPackM, pl = i / kPackM;
    const int m = m0 + ml, p = g * KW + pl;
    const bool act = m <= mmax && p < npair;
    const bool south = act && p != npair - 1;  // the equator ring has no mirror
    long long on = 0, os = 0;
    int kk = 0;
    bool conj = false;
    float2 en = make_float2(0.f, 0.f), es = en;
    if (act) {
      const RingInfo Rn = rings[p];
      const unsigned N = (unsigned)Rn.nphi, k = (unsigned)m % N, twoN = 2u * N;
      conj = k > (N >> 1);
      kk = (int)(conj ? N - k : k);
      on = Rn.specoff;  // sigma m < 2^15: the phase index in 32 bits
      en = cscale(etab[Rn.etab + ((unsigned)Rn.sigma * (unsigned)m) % twoN], use_w ? (float)Rn.w : 1.f);
      if (south) {  // mirror ring: same length, same table
        const RingInfo Rs = rings[nring - 1 - p];
        os = Rs.specoff;
        es = cscale(etab[Rs.etab + ((unsigned)Rs.sigma * (unsigned)m) % twoN], use_w ? (float)Rs.w : 1.f);
      }
    }
    E* T = reinterpret_cast<E*>(smem_raw + ml * slab) + pl;
    // all the item's spectrum bins first (16 loads in flight), then the operand values
    float2 xn[kPackC], xs[kPackC];
#pragma unroll
    for (int cl = 0; cl < kPackC; ++cl) {
      xn[cl] = xs[cl] = make_float2(0.f, 0.f);
      if (act && cl < nch) {
        const float2* X = spec + (long long)(b0 + c0 + cl) * nspec;
        xn[cl] = X[on + kk];
        if (south) xs[cl] = X[os + kk];
      }
    }
#pragma unroll
    for (int cl = 0; cl < kPackC; ++cl) {
      const float2 gn = cmul(conj ? cconj(xn[cl]) : xn[cl], en);
      const float2 gs = cmul(conj ? cconj(xs[cl]) : xs[cl], es);
      const float sc = csc[cl];
      const float v[4] = {(gn.x + gs.x) * sc, (gn.y + gs.y) * sc, (gn.x - gs.x) * sc, (gn.y - gs.y) * sc};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int r = (q >> 1) * 2 * kPackC + 2 * cl + (q & 1);  // S rows, then A rows
        const E h = Elt<E>::from_float(v[q]);
        T[r * KW] = h;
        if (x3) T[(r + 4 * kPackC) * KW] = Elt<E>::from_float(v[q] - Elt<E>::to_float(h));
      }
    }
  }
  __syncthreads();
  // local row rr: part rr / (2 kPackC) (S hi, A hi, S lo, A lo) at operand
  // row (A: + C2N) (lo: + NN) + 2 c0 + rr % (2 kPackC)
  for (int q = threadIdx.x; q < kPackM * rows * 8; q += blockDim.x) {
    const int ml = q / (rows * 8), rr = (q >> 3) % rows, ch = q & 7;
    const int m = m0 + ml;
    if (m > mmax) continue;
    const int part = rr / (2 * kPackC);
    const int grow = ((part & 1) ? C2N : 0) + ((part & 2) ? NN : 0) + 2 * c0 + rr % (2 * kPackC);
    const uint4 val = *reinterpret_cast<const uint4*>(smem_raw + ml * slab + rr * 128 + ch * 16);
    *reinterpret_cast<uint4*>(reinterpret_cast<unsigned char*>(gt) +
                              (((long long)m * ngroup + g) * rb + grow) * 128 + ch * 16) = val;
  }
}

// ---------------------------------------------------------------------------
// synthesis operand: At[chunk][rows][KW] from alm
// ---------------------------------------------------------------------------
// For l = m + KW j + (0..KW-1): row n < 2 CP holds part n%2 of
// s_c P_l mfac a_lm of channel n/2 where l - m is even (0 elsewhere), row
// 2 CP + n the same for odd l - m; zero past lmax; x3 remainders in rows
// NN .. 2 NN - 1.  Only Re a_l0 enters (real maps).
template <int CP, typename E>
__global__ void __launch_bounds__(128)
k_pack_at(const float2* __restrict__ alm, const float* __restrict__ coef_pf, const long long* __restrict__ achunk,
          E* __restrict__ at, int lmax, int mmax, long long nalm, int b0, int nb, float mfac, int x3,
          const unsigned* __restrict__ bmax, float sfac) {
  constexpr int KW = Elt<E>::kw, C2N = 2 * CP, NN = 2 * C2N;
  const int rb = x3 ? 2 * NN : NN;
  const int m = blockIdx.y, j = blockIdx.x * (128 / KW) + threadIdx.x / KW, lane = threadIdx.x % KW;
  if (m > mmax || j > (lmax - m) / KW) return;
  const int l = m + KW * j + lane;
  E* out = at + (achunk[m] + j) * rb * KW + lane;
  const bool in = l <= lmax;
  const bool odd = ((l - m) & 1) != 0;
  const long long base = alm_base(lmax, m);
  // P_l (FP32) times factors of two (mfac, the channel scale): exact
  const float s = in ? coef_pf[base + l] * (m > 0 ? mfac : 1.f) : 0.f;
#pragma unroll 8
  for (int c = 0; c < CP; ++c) {
    float2 a = make_float2(0.f, 0.f);
    if (in && c < nb) a = alm[(long long)(b0 + c) * nalm + base + l];
    if (in && c < nb) {
      const float sc = s * chan_scale(bmax, b0 + c, sfac);
      a = make_float2(sc * a.x, m == 0 ? 0.f : sc * a.y);
    }
    const float2 e = odd ? make_float2(0.f, 0.f) : a, o = odd ? a : make_float2(0.f, 0.f);
    put(out, 2 * c, NN, e.x, x3);
    put(out, 2 * c + 1, NN, e.y, x3);
    put(out, C2N + 2 * c, NN, o.x, x3);
    put(out, C2N + 2 * c + 1, NN, o.y, x3);
  }
}

// ---------------------------------------------------------------------------
// plan-time lambda tables of the tensor-core stages
// ---------------------------------------------------------------------------
// The recurrence of every table: the FP32 plans' chain (Recur<float>, the
// same steps as the CUDA-core kernels', so FP32 tables hold identical
// values), from l = ls, restarted at the chain start lc with the stored
// (mu_{lc-1}, mu_lc); zero before lc.  16-bit tables hold kLamScale mu: the
// restart values scaled by that power of two scale every later value
// exactly.
struct Chain {
  Recur<float> rc;
  int lc;
  const float2* c;
  __device__ __forceinline__ float step(int l) { return rc.step(c[l], l, lc); }
};
template <typename E>
__device__ __forceinline__ Chain chain_at(const RingInfo* rings, const float2* coef_cf, const int* lc_tab,
                                          const double* mu0_tab, const double* mu1_tab, int lmax, int npair, int m,
                                          int p) {
  Chain ch;
  ch.lc = INT_MAX;
  ch.c = coef_cf + alm_base(lmax, m);
  if (p < npair) {
    const long long ci = (long long)m * npair + p;
    constexpr double kS = sizeof(E) == 2 ? kLamScale : 1.0;
    ch.lc = lc_tab[ci];
    ch.rc.start(rings[p].z, kS * mu0_tab[ci], kS * mu1_tab[ci]);
  }
  return ch;
}
// A table value as a stored element and its remainder: hi the FP32 value
// rounded to E, lo the remainder (exact in FP32) rounded to E; hi + lo is
// within 2^-22 |value| for 16-bit E.  FP32 tables store the value alone.
template <typename E>
__device__ __forceinline__ void split_value(float f, E& hi, E& lo) {
  hi = Elt<E>::from_float(f);
  lo = Elt<E>::from_float(f - Elt<E>::to_float(hi));
}

// Row table (analysis) of 16-bit types: per (m, group of KW = 64 pairs), rows
// l = ls_g .. lmax of 64 values, ls_g the group's first significant l aligned
// down to the analysis tile grid m + 128 j.  (The FP32 row table, in groups
// of 32 pairs, is the CUDA-core kernels' table.)
__global__ void k_rtab_groups(const int* __restrict__ lc_tab, int lmax, int npair, int kw, int ngroup, int* lstart,
                              long long* rows) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x, m = blockIdx.y;
  if (g >= ngroup) return;
  int ls = lmax + 1;
  for (int j = 0; j < kw; ++j) {
    const int p = g * kw + j;
    if (p < npair) ls = min(ls, lc_tab[(long long)m * npair + p]);
  }
  if (ls <= lmax) ls = m + ((ls - m) / kTcTile) * kTcTile;
  lstart[(long long)m * ngroup + g] = ls;
  rows[(long long)m * ngroup + g] = lmax + 1 - ls;
}

// Fills m = m0 + blockIdx.y; element e of the table goes to hi[e - base]
// (base > 0 when the table is built block by block through a staging buffer).
template <typename E>
__global__ void k_rtab_fill(const RingInfo* __restrict__ rings, const float2* __restrict__ coef_c,
                            const int* __restrict__ lc_tab, const double* __restrict__ mu0_tab,
                            const double* __restrict__ mu1_tab, const int* __restrict__ lstart,
                            const long long* __restrict__ off, int lmax, int npair, int ngroup, int m0,
                            long long base, E* hi, E* lo) {
  constexpr int KW = Elt<E>::kw;
  const int p = blockIdx.x * blockDim.x + threadIdx.x, m = m0 + blockIdx.y;
  const int g = p / KW;
  if (g >= ngroup) return;
  const long long mg = (long long)m * ngroup + g;
  const int ls = lstart[mg];
  const long long o = off[mg] - base + (p % KW);
  Chain ch = chain_at<E>(rings, coef_c, lc_tab, mu0_tab, mu1_tab, lmax, npair, m, p);
  // rows before the warp's first chain start are zero: no recurrence there
  // (a group's warps are whole, so the early return above left all lanes)
  const int lw = min(__reduce_min_sync(0xffffffffu, ch.lc), lmax + 1);
  int l = ls;
  for (; l < lw; ++l) {
    hi[o + (long long)(l - ls) * KW] = Elt<E>::from_float(0.f);
    if (lo) lo[o + (long long)(l - ls) * KW] = Elt<E>::from_float(0.f);
  }
  for (; l <= lmax; ++l) {
    E h, r;
    split_value<E>(p < npair ? ch.step(l) : 0.f, h, r);
    hi[o + (long long)(l - ls) * KW] = h;
    if (lo) lo[o + (long long)(l - ls) * KW] = r;
  }
}

// Column table (synthesis): per (m, tile T of 128 ring pairs), from ls_T =
// the tile's first significant l (aligned down to m + KW j) to lmax, blocks
// of 128 pairs x KW l, element [p][l] (zero before a chain's start, past lmax
// and for pairs past npair).
__global__ void k_ctab_tiles(const int* __restrict__ lc_tab, int lmax, int npair, int kw, int nptile, int* lstart,
                             long long* nblk) {
  const int T = blockIdx.x * blockDim.x + threadIdx.x, m = blockIdx.y;
  if (T >= nptile) return;
  int ls = lmax + 1;
  for (int j = 0; j < 128; ++j) {
    const int p = T * 128 + j;
    if (p < npair) ls = min(ls, lc_tab[(long long)m * npair + p]);
  }
  if (ls <= lmax) ls = m + ((ls - m) / kw) * kw;
  lstart[(long long)m * nptile + T] = ls;
  nblk[(long long)m * nptile + T] = ls <= lmax ? (lmax - ls) / kw + 1 : 0;
}

template <typename E>
__global__ void k_ctab_fill(const RingInfo* __restrict__ rings, const float2* __restrict__ coef_c,
                            const int* __restrict__ lc_tab, const double* __restrict__ mu0_tab,
                            const double* __restrict__ mu1_tab, const int* __restrict__ lstart,
                            const long long* __restrict__ off, int lmax, int npair, int nptile, int m0,
                            long long base, E* hi, E* lo) {
  constexpr int KW = Elt<E>::kw, V = 16 / (int)sizeof(E);  // values per 16-byte store
  const int p = blockIdx.x * blockDim.x + threadIdx.x, m = m0 + blockIdx.y;
  const int T = p >> 7;
  if (T >= nptile) return;
  const long long mT = (long long)m * nptile + T;
  const int ls = lstart[mT];
  if (ls > lmax) return;
  const int lend = ls + ((lmax - ls) / KW + 1) * KW;  // end of the last block
  const long long o = off[mT] - base + (long long)(p & 127) * KW;
  Chain ch = chain_at<E>(rings, coef_c, lc_tab, mu0_tab, mu1_tab, lmax, npair, m, p);
  // vectors wholly before the warp's first chain start are zero: no
  // recurrence there (a tile's warps are whole: the early returns above
  // take all 128 threads of a tile or none)
  const int lw = __reduce_min_sync(0xffffffffu, ch.lc);
  for (int lv = ls; lv < lend; lv += V) {
    alignas(16) E h[V];
    alignas(16) E r[V];
    if (lv + V <= lw) {
#pragma unroll
      for (int u = 0; u < V; ++u) h[u] = r[u] = Elt<E>::from_float(0.f);
    } else {
#pragma unroll
      for (int u = 0; u < V; ++u) {
        const int l = lv + u;
        split_value<E>((l <= lmax && p < npair) ? ch.step(l) : 0.f, h[u], r[u]);
      }
    }
    const int q = lv - ls;
    const long long at = o + (long long)(q / KW) * 128 * KW + (q % KW);
    *reinterpret_cast<uint4*>(hi + at) = *reinterpret_cast<const uint4*>(h);
    if (lo) *reinterpret_cast<uint4*>(lo + at) = *reinterpret_cast<const uint4*>(r);
  }
}

// ---------------------------------------------------------------------------
// the tile kernel
// ---------------------------------------------------------------------------
// MODE 0: FP32 operands, 3xTF32 with the remainders made in shared memory;
// MODE 1: one 16-bit product; MODE 2: 16-bit x3 (stored hi and lo parts).
__host__ __device__ constexpr int pow2_at_least(int x) { return x <= 32 ? 32 : 2 * pow2_at_least((x + 1) / 2); }

// m per CTA of the single-product synthesis of 64 channels (N = 256): 2,
// whose outputs fill the 512 tensor-memory columns (one CTA per SM), F
// leaving in 16-byte pieces.
#ifndef HPX_TC_SYN_MQ_256
#define HPX_TC_SYN_MQ_256 2
#endif
// ... and of 32 channels (N = 128): 4, again all 512 columns, so that F
// leaves in whole 32-byte sectors (at Nside 1024 / lmax 2047 / 64 BF16
// channels 4.13 ms against 5.77 with 64 channels per CTA and 5.92 with 2 m).
#ifndef HPX_TC_SYN_MQ_128
#define HPX_TC_SYN_MQ_128 4
#endif
// m per CTA of the split-product synthesis of 16 channels (N = 64): 2 (two
// CTAs per SM); 4 fills the tensor memory and measured slower (10.5 against
// 9.0 ms at the same workload in FP32).
#ifndef HPX_TC_SYN_MQ_X3
#define HPX_TC_SYN_MQ_X3 2
#endif

template <int NN, bool SYN, int MODE>
struct TcShape {
  static constexpr int kA = kTcTile * 128;  // lambda tile bytes: 128 rows x 128 bytes
  static constexpr int kG = NN * 128;       // B tile bytes (Gt or At)
  static constexpr int kStage = MODE == 0 ? kA + 2 * kG : MODE == 1 ? kA + kG : 2 * kA + 2 * kG;
  // MODE 0: the lambda remainders go to tensor memory (32 columns per K
  // block, two buffers) where that keeps the CTA within 256 columns (N = 32),
  // else to two shared-memory buffers
  static constexpr bool kLoTmem = MODE == 0 && NN == 32;
  static constexpr int kLo = MODE == 0 && !kLoTmem ? kA : 0;
  static constexpr int kBuf = MODE == 0 ? 2 * NN : NN;  // TMEM columns of one block accumulator
  static constexpr int kLoCol = 2 * kBuf;                // first TMEM column of the remainder buffers
  // MODE 1 (one 16-bit product, error bounds of 1e-2 / 2e-3): each m
  // accumulates over its whole K range in its own TMEM region, drained once
  // (the accumulator's truncation, ~1e-6, is far inside those bounds); the
  // other modes accumulate each K block alone and add it into FP32 registers
  static constexpr bool kFullK = MODE == 1;
  // synthesis m per CTA (see tc_mq)
  static constexpr int kMq =
      (SYN && MODE != 0)
          ? (kFullK ? (NN <= 64 ? 4 : NN == 256 ? HPX_TC_SYN_MQ_256 : HPX_TC_SYN_MQ_128)
                    : (NN == 32 ? 4 : NN == 64 ? HPX_TC_SYN_MQ_X3 : 2))
          : 1;
  static constexpr int kTmemCols = kFullK ? pow2_at_least(kMq * NN) : kLoTmem ? 256 : 2 * kBuf;
  static constexpr int kAlloc = (!kFullK && kMq > 1) ? pow2_at_least(kTmemCols + kMq * NN) : kTmemCols;
  // two CTAs per SM where half the tensor memory and half the shared memory
  // (with at least two stages) suffice: the second CTA's prologue, tail and
  // epilogue then overlap the first's streaming
  static constexpr int kStages2 = (110 * 1024 - 2 * kLo) / kStage;
  static constexpr int kCtas = (kAlloc <= 256 && kStages2 >= 2 && (NN <= 64 || kFullK)) ? 2 : 1;
  static constexpr int kBudget = kCtas == 2 ? 110 * 1024 : 200 * 1024;
  static constexpr int kNStage = (kBudget - 2 * kLo) / kStage < 8 ? (kBudget - 2 * kLo) / kStage : 8;
  static constexpr size_t kSmem =
      (size_t)kNStage * kStage + 2 * kLo + 1024 /* base alignment */ + 2048 /* barriers, lists */;
  static_assert(kNStage >= 2 && kTmemCols <= 512 && kTmemCols >= 32, "shape");
  static_assert(!kLoTmem || kLoCol + 64 <= kTmemCols, "remainder buffers inside the allocation");
};

constexpr int kTcThreads = 192;  // warps 0-3 split and drain, warp 4 copies, warp 5 issues products

// Synthesis CTAs of the 16-bit modes take kMq consecutive m of one pair tile:
// each finished m's outputs wait in spare tensor-memory columns, so that the
// epilogue writes every ring's kMq values of F (m fastest) as one piece --
// whole 32-byte sectors at kMq = 4 -- instead of one 8-byte value per CTA.
// kMq NN staging columns fit beside the accumulators within the allocation.
template <int NN, bool SYN, int MODE>
__host__ __device__ constexpr int tc_mq() {
  return TcShape<NN, SYN, MODE>::kMq;
}

struct TcArgs {
  const long long* off;     // analysis: row table offsets [m][group]; synthesis: column table [m][p tile]
  const int* lstart;        // first l stored, same indexing
  int ngroup;               // groups (analysis) or p tiles (synthesis) per m
  const long long* achunk;  // synthesis: first At chunk of each m
  const float* coef_pf;     // analysis: P_l (FP32)
  const unsigned* bmax;     // 16-bit operands: per-channel largest component
  float sfac;               // bound factor for the channel scale
  float lscale;             // 1 / the table's lambda scale
  float* out;               // analysis: alm [b][nalm] complex; synthesis: F [b][nring][mmax+1] complex
  int lmax, mmax, npair, nring;
  long long nalm;
  int b0, nb;
  double mfac;
  uint32_t fmt;             // 16-bit modes: operand format of kind::f16 (0 FP16, 1 BF16)
  int* status;
  int m0, nm;               // the launch's m range (analysis: blockIdx.y = m - m0)
  long long tbase;          // table element at row 0 of the lambda descriptor (streamed blocks)
  int withhold;             // test support: issue no copies, so the first wait for one runs out
  int ncg;                  // synthesis: channel groups of the launch (CTAs per pair tile)
  long long cg_rows;        // synthesis: operand rows between consecutive groups' At regions
};

// One CTA: a 128-row tile of one m, all channels of the launch.
//   analysis (SYN false): rows are l = l0 .. l0+127, K runs over the KW-pair
//     groups whose table rows reach the tile, B = Gt: D[l][n] = sum_p L G;
//   synthesis (SYN true): rows are ring pairs p = 128 T .. 128 T + 127, K runs
//     over KW-l chunks from the tile's first significant l, A = the column
//     table's blocks, B = At: D[p][n] = sum_l L^T At.
// Per K block k, with L the lambda tile (128 x KW) and B (NN x KW) in shared
// memory, in 4 instruction steps of 32 bytes along K:
//   MODE 0: lo(L), lo(B) are formed (hi is the hardware's TF32 truncation of
//           the tile as loaded; lo = x - trunc(x), rounded to TF32); lo(B)
//           sits right after B, so D[:, 0:2NN] += L [B; lo B]^T and
//           D[:, 0:NN] += lo(L) B^T (2 instructions per step); the drain
//           adds D[r][j] + D[r][NN + j];
//   MODE 1: D += L B^T;  MODE 2: D += L B^T + L lo(B)^T + lo(L) B^T, with
//           lo(L) and lo(B) loaded next to L and B.
// The drain keeps the NN/2 columns of the row's parity (analysis) or all NN
// (synthesis) and adds them into FP32 registers (round to nearest).  The
// tensor cores add each instruction's products into the accumulator with
// truncation, so each block is accumulated alone, in one of two TMEM
// buffers, while the other is drained.
//
// Roles run decoupled, linked by mbarriers: warp 4 keeps up to kNStage
// blocks of copies in flight, warp 5 issues a block's products once it has
// landed (and, MODE 0, is split) and its accumulator is free, warps 0-3 split
// block k (MODE 0) and drain block k-1.  After an expired wait a role stops
// working (the split/drain warps keep looping without work, so their
// warp-collective tcgen05.ld stays convergent), waits for what it started,
// and the CTA records the timeout.
template <int NN, bool SYN, int MODE>
__global__ void __launch_bounds__(kTcThreads, TcShape<NN, SYN, MODE>::kCtas)
k_legendre_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmAlo,
              const __grid_constant__ CUtensorMap tmB, const TcArgs a) {
  using S = TcShape<NN, SYN, MODE>;
  constexpr bool FK = S::kFullK;
  constexpr int NS = S::kNStage, C2N = NN / 2, KW = MODE == 0 ? 32 : 64;
  constexpr int RB = MODE == 2 ? 2 * NN : NN;  // operand rows per K block in memory
  constexpr int NSUM = SYN ? NN : C2N;
  constexpr int MQ = tc_mq<NN, SYN, MODE>();
  constexpr int kStageCol = S::kTmemCols;  // first staging column (MQ > 1, not FK)
  constexpr int kAlloc = S::kAlloc;
  static_assert(kAlloc <= (S::kCtas == 2 ? 256 : 512), "tensor memory");
  static_assert(NN % 32 == 0 && NN <= (MODE == 0 || (SYN && !FK) ? 128 : 256), "N tile");
  static_assert(MQ <= 4, "per-m lists hold 4 entries");
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  // analysis: m; synthesis: the first of the CTA's nq consecutive m
  const int m = a.m0 + blockIdx.y * MQ;
  // the ncg channel groups of one tile (pairs: synthesis; l: analysis) are
  // consecutive CTAs, so they stream the same lambda blocks at about the same
  // time and all but the first read them from L2
  const int ptile = (int)blockIdx.x / a.ncg;
  const int cgi = (int)blockIdx.x % a.ncg;
  const int b0 = a.b0 + cgi * (C2N / 2);           // first channel of the CTA
  const int nbl = min(C2N / 2, a.nb - cgi * (C2N / 2));  // its channels
  const int nq = SYN ? min(MQ, a.m0 + a.nm - m) : 1;
  const int l0 = m + kTcTile * ptile;  // analysis tile
  if (!SYN && l0 > a.lmax) return;          // whole CTA, before any shared state

  extern __shared__ unsigned char smem_raw[];
  unsigned char* tiles = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* lobuf = tiles + (size_t)NS * S::kStage;
  uint64_t* full = reinterpret_cast<uint64_t*>(lobuf + 2 * S::kLo);
  uint64_t* conv = full + NS;   // stage split (128 arrivals; MODE 0)
  uint64_t* empty = conv + NS;  // stage's products done
  uint64_t* accf = empty + NS;  // [2] block accumulator complete
  uint64_t* acce = accf + 2;    // [2] block accumulator drained (128 arrivals)
  uint64_t* done = acce + 2;    // all products done
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  int* wcount = reinterpret_cast<int*>(tmem_slot + 2);  // [4]
  int* rowA = wcount + 4;   // analysis: [128] TMA row of the lambda tile of active group k
  int* rowB = rowA + 128;   // analysis: [128] TMA row of its operand tile
  int* qna = rowB + 128;    // synthesis: [MQ] blocks, first lambda row, first operand row of each m
  int* qra = qna + 4;
  int* qrb = qra + 4;
  auto sL = [&](int s) { return tiles + (size_t)s * S::kStage; };
  auto sB = [&](int s) { return tiles + (size_t)s * S::kStage + (MODE == 2 ? 2 : 1) * S::kA; };
  auto sBlo = [&](int s) { return tiles + (size_t)s * S::kStage + (MODE == 2 ? 2 : 1) * S::kA + S::kG; };
  auto sLlo = [&](int s, int b) {
    return MODE == 2 ? tiles + (size_t)s * S::kStage + S::kA : lobuf + (size_t)b * S::kLo;
  };

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kAlloc));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  // K blocks.  Analysis: groups whose rows reach this tile (group starts lie
  // on the tile grid m + 128 j, so a group covers the whole tile or starts
  // after it), with their copy coordinates, compacted in group order.
  // Synthesis: every KW-l chunk from the tile's first stored l.
  bool act = false;
  int ra = 0, rb = 0;
  unsigned bal = 0;
  if (!SYN && warp < 4) {
    if (t < a.ngroup) {
      const long long mg = (long long)m * a.ngroup + t;
      const int ls = a.lstart[mg];
      act = ls <= l0;
      ra = (int)((a.off[mg] - a.tbase) / KW) + (l0 - ls);
      rb = (int)(mg * RB + cgi * a.cg_rows);
    }
    bal = __ballot_sync(0xffffffffu, act);
    if (lane == 0) wcount[warp] = __popc(bal);
  }
  int na = 0;  // K blocks of the CTA
  if (SYN && warp == 1 && lane < MQ) {  // synthesis: per m of the CTA, its block count and first rows
    int n = 0, ra = 0, rb = 0;
    if (lane < nq) {
      const int mj = m + lane;
      const long long mT = (long long)mj * a.ngroup + ptile;
      const int ls = a.lstart[mT];
      if (ls <= a.lmax) {
        n = (a.lmax - ls) / KW + 1;
        ra = (int)((a.off[mT] - a.tbase) / KW);
        rb = (int)((a.achunk[mj] + (ls - mj) / KW) * RB + cgi * a.cg_rows);
      }
    }
    qna[lane] = n;
    qra[lane] = ra;
    qrb[lane] = rb;
  }
  if (t == 32) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&conv[s], 128);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {  // FK: accf[0..3] (acce follows accf), one arrival each
      mbar_init(&accf[b], 1);
      mbar_init(&acce[b], FK ? 1 : 128);
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
  } else {
    for (int j = 0; j < MQ; ++j) na += qna[j];
  }
  const uint32_t tmem = *tmem_slot;
  __syncthreads();

  if (warp == 4) {
    // ---- copies: block k into stage k % NS once block k - NS's products are done
    int issued = 0;
    if (lane == 0 && !a.withhold) {
      constexpr uint32_t kBytes = MODE == 2 ? 2 * (S::kA + S::kG) : S::kA + S::kG;
      int j = 0, kj = 0;  // synthesis: m of the CTA and block within it
      for (int k = 0; k < na; ++k) {
        const int s = k % NS;
        if (k >= NS && !wait_phase(&empty[s], (uint32_t)(k / NS - 1) & 1u, abort_flag, true)) break;
        if (SYN)
          while (kj >= qna[j]) {
            kj = 0;
            ++j;
          }
        const int r_a = SYN ? qra[j] + kj * 128 : rowA[k], r_b = SYN ? qrb[j] + kj * RB : rowB[k];
        ++kj;
        mbar_expect_tx(&full[s], kBytes);
        tma_load_2d(sL(s), &tmA, 0, r_a, &full[s]);
        tma_load_2d(sB(s), &tmB, 0, r_b, &full[s]);
        if (MODE == 2) {
          tma_load_2d(sLlo(s, 0), &tmAlo, 0, r_a, &full[s]);
          tma_load_2d(sBlo(s), &tmB, 0, r_b + NN, &full[s]);
        }
        issued = k + 1;
      }
      // whatever was started completes before the CTA moves on
      for (int k = issued > NS ? issued - NS : 0; k < issued; ++k)
        wait_phase(&full[k % NS], (uint32_t)(k / NS) & 1u, abort_flag, false);
    }
  } else if (warp == 5) {
    // ---- products
    if (lane == 0) {
      // instruction descriptors: D f32, A and B K-major, M = 128; tf32 (2)
      // or the 16-bit format
      const uint32_t f = MODE == 0 ? 2u : a.fmt;
      const uint32_t id2 = (1u << 4) | (f << 7) | (f << 10) | ((uint32_t)(2 * NN >> 3) << 17) | ((128u >> 4) << 24);
      const uint32_t id1 = (1u << 4) | (f << 7) | (f << 10) | ((uint32_t)(NN >> 3) << 17) | ((128u >> 4) << 24);
      bool issued_any = false;
      if constexpr (FK) {
        // every block of the CTA's j-th m accumulates into TMEM region j;
        // accf[j] completes once the products of its last block have
        int j = 0, kj = 0;
        for (int k = 0; k < na; ++k) {
          const int s = k % NS;
          if constexpr (SYN)
            while (kj >= qna[j]) {
              kj = 0;
              ++j;
            }
          if (!wait_phase(&full[s], (uint32_t)(k / NS) & 1u, abort_flag, true)) break;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t d = tmem + (uint32_t)(j * NN);
          const uint32_t aL = smem_u32(sL(s)), aB = smem_u32(sB(s));
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const uint32_t off = 32u * q;
            umma_f16(d, sdesc_sw128(aL + off), sdesc_sw128(aB + off), id1, (kj > 0 || q > 0) ? 1u : 0u);
          }
          umma_commit(&empty[s]);
          ++kj;
          if (kj == (SYN ? qna[j] : na)) umma_commit(&accf[j]);
          issued_any = true;
        }
      } else
      for (int k = 0; k < na; ++k) {
        const int s = k % NS, b = k & 1;
        if (!wait_phase(MODE == 0 ? &conv[s] : &full[s], (uint32_t)(k / NS) & 1u, abort_flag, true)) break;
        if (k >= 2 && !wait_phase(&acce[b], (uint32_t)((k - 2) >> 1) & 1u, abort_flag, true)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t d = tmem + (uint32_t)(b * S::kBuf);
        const uint32_t aL = smem_u32(sL(s)), aLlo = smem_u32(sLlo(s, b)), aB = smem_u32(sB(s)),
                       aBlo = smem_u32(sBlo(s));
#pragma unroll
        for (int j = 0; j < 4; ++j) {  // 32 bytes along K per instruction (8 tf32 or 16 16-bit values)
          const uint32_t off = 32u * j;
          if constexpr (MODE == 0) {
            umma_tf32(d, sdesc_sw128(aL + off), sdesc_sw128(aB + off), id2, j > 0 ? 1u : 0u);
            if constexpr (S::kLoTmem)  // lo(L) from tensor memory: lane = row, 8 columns per step
              umma_tf32_ta(d, tmem + (uint32_t)(S::kLoCol + b * 32 + 8 * j), sdesc_sw128(aB + off), id1, 1u);
            else
              umma_tf32(d, sdesc_sw128(aLlo + off), sdesc_sw128(aB + off), id1, 1u);
          } else {
            umma_f16(d, sdesc_sw128(aL + off), sdesc_sw128(aB + off), id1, j > 0 ? 1u : 0u);
            if constexpr (MODE == 2) {
              umma_f16(d, sdesc_sw128(aL + off), sdesc_sw128(aBlo + off), id1, 1u);
              umma_f16(d, sdesc_sw128(aLlo + off), sdesc_sw128(aB + off), id1, 1u);
            }
          }
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
    auto col = [&](const uint32_t* v1, const uint32_t* v2, int j) {
      return MODE == 0 ? __uint_as_float(v1[j]) + __uint_as_float(v2[j]) : __uint_as_float(v1[j]);
    };
    auto drain = [&](int buf) {  // warp-collective
      const uint32_t c0 = trow + (uint32_t)(buf * S::kBuf);
      if constexpr (MODE != 0) {
        // 16-bit modes: QB loads of 16 columns in flight per wait (the
        // accumulator read back in few round trips)
        constexpr int NQ = SYN ? NN / 16 : C2N / 16;
        constexpr int QB = SYN ? (NQ < 4 ? NQ : 4) : (NQ < 2 ? NQ : 2);
#pragma unroll
        for (int q0 = 0; q0 < NQ; q0 += QB) {
          uint32_t v1[QB][16], v2[SYN ? 1 : QB][16];
#pragma unroll
          for (int u = 0; u < QB; ++u) {
            tmem_ld16(c0 + (uint32_t)((q0 + u) * 16), v1[u]);
            if constexpr (!SYN) tmem_ld16(c0 + (uint32_t)(C2N + (q0 + u) * 16), v2[u]);
          }
          tmem_wait_ld();
#pragma unroll
          for (int u = 0; u < QB; ++u)
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              if constexpr (SYN)
                sum[(q0 + u) * 16 + j] += __uint_as_float(v1[u][j]);
              else
                sum[(q0 + u) * 16 + j] += __uint_as_float(odd ? v2[u][j] : v1[u][j]);
            }
        }
      } else if constexpr (SYN) {
#pragma unroll
        for (int q = 0; q < NN / 16; ++q) {
          uint32_t v1[16], v2[16];
          tmem_ld16(c0 + (uint32_t)(q * 16), v1);
          tmem_ld16(c0 + (uint32_t)(NN + q * 16), v2);
          tmem_wait_ld();
#pragma unroll
          for (int j = 0; j < 16; ++j) sum[q * 16 + j] += col(v1, v2, j);
        }
      } else {
#pragma unroll
        for (int q = 0; q < C2N / 16; ++q) {
          uint32_t s1[16], s2[16], a1[16], a2[16];
          tmem_ld16(c0 + (uint32_t)(q * 16), s1);
          tmem_ld16(c0 + (uint32_t)(C2N + q * 16), a1);
          tmem_ld16(c0 + (uint32_t)(NN + q * 16), s2);
          tmem_ld16(c0 + (uint32_t)(NN + C2N + q * 16), a2);
          tmem_wait_ld();
#pragma unroll
          for (int j = 0; j < 16; ++j) sum[q * 16 + j] += odd ? col(a1, a2, j) : col(s1, s2, j);
        }
      }
    };
    // synthesis with several m per CTA (MQ > 1): when all blocks of the next
    // m are drained, its outputs go to staging columns and the sums restart
    int jn = 0, jend = 0;  // next m to finish; blocks before it
    auto finish = [&]() {  // warp-collective
      if constexpr (MQ > 1) {
#pragma unroll
        for (int g = 0; g < NN / 32; ++g) {  // 8 channels: north re, im, south re, im each
          uint32_t v[32];
#pragma unroll
          for (int cc = 0; cc < 8; ++cc) {
            const int c = 8 * g + cc;
            const float inv = a.lscale / chan_scale(a.bmax, b0 + c, a.sfac);  // a power of two
            const float er = sum[2 * c] * inv, ei = sum[2 * c + 1] * inv;
            const float orr = sum[C2N + 2 * c] * inv, oi = sum[C2N + 2 * c + 1] * inv;
            v[4 * cc] = __float_as_uint(er + orr);
            v[4 * cc + 1] = __float_as_uint(ei + oi);
            v[4 * cc + 2] = __float_as_uint(er - orr);
            v[4 * cc + 3] = __float_as_uint(ei - oi);
          }
          tmem_st32(trow + (uint32_t)(kStageCol + jn * NN + 32 * g), v);
        }
#pragma unroll
        for (int j = 0; j < NSUM; ++j) sum[j] = 0.f;
        ++jn;
      }
    };
    auto advance = [&](int drained) {  // `drained` blocks of the CTA are in the sums
      if constexpr (MQ > 1) {
        while (jn < MQ && jend + qna[jn] <= drained) {
          jend += qna[jn];
          finish();
        }
      }
    };
    if constexpr (FK) {
      // one wait for the CTA's products: accf of its last m with blocks (a
      // commit tracks every product the issuing thread started before it)
      int last = -1;
      if constexpr (SYN) {
        for (int j = 0; j < MQ; ++j)
          if (qna[j] > 0) last = j;
      } else {
        last = na > 0 ? 0 : -1;
      }
      if (last >= 0) {
        bool ok = wait_phase(&accf[last], 0u, abort_flag, true);
        ok = __all_sync(0xffffffffu, ok);
        if (ok) asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      }
    } else {
      advance(0);  // leading m without blocks
      bool alive = true;
      for (int k = 0; k < na; ++k) {
        const int s = k % NS, b = k & 1;
        if (MODE == 0) {
          if (alive) alive = wait_phase(&full[s], (uint32_t)(k / NS) & 1u, abort_flag, true);
          if constexpr (S::kLoTmem) alive = __all_sync(0xffffffffu, alive);  // the TMEM store is warp-collective
          if (alive) {
            // elementwise, so the swizzle does not matter; consecutive threads
            // take consecutive 16-byte words.  Remainder buffer b was last read
            // by block k-2's products, complete since this thread drained that
            // block in the previous iteration.
            if constexpr (S::kLoTmem) {
              // this thread's row t of the tile (128 bytes, 16-byte chunks
              // permuted by the swizzle: chunk c at c ^ (t mod 8)) to TMEM lane t
              const unsigned char* row = sL(s) + t * 128;
              uint32_t v[32];
  #pragma unroll
              for (int c = 0; c < 8; ++c) {
                const float4 q = tf32_rem4(*reinterpret_cast<const float4*>(row + ((c ^ (t & 7)) << 4)));
                v[4 * c] = __float_as_uint(q.x);
                v[4 * c + 1] = __float_as_uint(q.y);
                v[4 * c + 2] = __float_as_uint(q.z);
                v[4 * c + 3] = __float_as_uint(q.w);
              }
              tmem_st32(trow + (uint32_t)(S::kLoCol + b * 32), v);
            } else {
              const float4* x = reinterpret_cast<const float4*>(sL(s));
              float4* xlo = reinterpret_cast<float4*>(sLlo(s, b));
  #pragma unroll
              for (int j = 0; j < S::kA / 2048; ++j) xlo[j * 128 + t] = tf32_rem4(x[j * 128 + t]);
            }
            const float4* y = reinterpret_cast<const float4*>(sB(s));
            float4* ylo = reinterpret_cast<float4*>(sBlo(s));
  #pragma unroll
            for (int j = 0; j < S::kG / 2048; ++j) ylo[j * 128 + t] = tf32_rem4(y[j * 128 + t]);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            if constexpr (S::kLoTmem) asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            mbar_arrive(&conv[s]);
          }
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
          advance(k);
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
      advance(na);
    }
    __syncwarp();
    // the CTA-wide sync below orders these writes after every role finished;
    // results are written only if no wait expired anywhere in the CTA
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (*abort_flag == 0) {
      if constexpr (FK && SYN) {
        // region j: E (columns 0 .. C2N-1) and O (C2N .. NN-1) of the CTA's
        // j-th m (zero if it had no blocks); north ring p gets E + O, its
        // mirror E - O, a ring's nq values adjacent in F
        const int p = ptile * 128 + t;
        const int ys = p == a.npair - 1 ? -1 : a.nring - 1 - p;
        float2* F = reinterpret_cast<float2*>(a.out);
        const long long mstride = a.mmax + 1;
#pragma unroll 1
        for (int cg = 0; cg < C2N / 16; ++cg) {  // 8 channels: 16 E and 16 O columns
          uint32_t e[MQ][16], o[MQ][16];
#pragma unroll
          for (int j = 0; j < MQ; ++j) {
            tmem_ld16(trow + (uint32_t)(j * NN + 16 * cg), e[j]);
            tmem_ld16(trow + (uint32_t)(j * NN + C2N + 16 * cg), o[j]);
          }
          tmem_wait_ld();
#pragma unroll
          for (int cc = 0; cc < 8; ++cc) {
            const int c = 8 * cg + cc;
            if (p < a.npair && c < nbl) {
              const float inv = a.lscale / chan_scale(a.bmax, b0 + c, a.sfac);  // a power of two
#pragma unroll
              for (int side = 0; side < 2; ++side) {
                const int y = side ? ys : p;
                if (y < 0) continue;
                const long long at = ((long long)(b0 + c) * a.nring + y) * mstride + m;
                float2 w[MQ];
#pragma unroll
                for (int j = 0; j < MQ; ++j) {
                  const bool has = qna[j] > 0;
                  const float er = has ? __uint_as_float(e[j][2 * cc]) * inv : 0.f;
                  const float ei = has ? __uint_as_float(e[j][2 * cc + 1]) * inv : 0.f;
                  const float orr = has ? __uint_as_float(o[j][2 * cc]) * inv : 0.f;
                  const float oi = has ? __uint_as_float(o[j][2 * cc + 1]) * inv : 0.f;
                  w[j] = side ? make_float2(er - orr, ei - oi) : make_float2(er + orr, ei + oi);
                }
                if (MQ % 2 == 0 && nq == MQ && (at % MQ) == 0) {  // whole pieces: 16 or 32 bytes
                  float4* dd = reinterpret_cast<float4*>(F + at);
#pragma unroll
                  for (int h = 0; h < MQ / 2; ++h)
                    dd[h] = make_float4(w[2 * h].x, w[2 * h].y, w[2 * h + 1].x, w[2 * h + 1].y);
                } else {
                  for (int j = 0; j < nq; ++j) F[at + j] = w[j];
                }
              }
            }
          }
        }
      } else if constexpr (FK) {
        // the row's own parity: A columns for odd l - m, S columns for even
        const long long base = alm_base(a.lmax, m);
        const bool row = l <= a.lmax && na > 0;
        const float scale = l <= a.lmax ? a.coef_pf[base + l] * (m > 0 ? (float)a.mfac : 1.f) * a.lscale : 0.f;
        float2* out = reinterpret_cast<float2*>(a.out) + (long long)b0 * a.nalm + base + l;
#pragma unroll 1
        for (int cg = 0; cg < C2N / 16; ++cg) {
          uint32_t sv[16], av[16];
          tmem_ld16(trow + (uint32_t)(16 * cg), sv);
          tmem_ld16(trow + (uint32_t)(C2N + 16 * cg), av);
          tmem_wait_ld();
#pragma unroll
          for (int cc = 0; cc < 8; ++cc) {
            const int c = 8 * cg + cc;
            if (l <= a.lmax && c < nbl) {
              const float inv = 1.f / chan_scale(a.bmax, b0 + c, a.sfac);
              const float re = row ? __uint_as_float(odd ? av[2 * cc] : sv[2 * cc]) : 0.f;
              const float im = row ? __uint_as_float(odd ? av[2 * cc + 1] : sv[2 * cc + 1]) : 0.f;
              out[(long long)c * a.nalm] = make_float2(scale * re * inv, scale * im * inv);
            }
          }
        }
      } else if constexpr (SYN && MQ > 1) {
        // the staged outputs of the CTA's nq m, 4 channels (16 columns) at a
        // time; per ring and channel the nq values are adjacent in F
        const int p = ptile * 128 + t;
        const int ys = p == a.npair - 1 ? -1 : a.nring - 1 - p;
        float2* F = reinterpret_cast<float2*>(a.out);
        const long long mstride = a.mmax + 1;
#pragma unroll
        for (int cg = 0; cg < NN / 16; ++cg) {
          uint32_t v[MQ][16];
#pragma unroll
          for (int j = 0; j < MQ; ++j) tmem_ld16(trow + (uint32_t)(kStageCol + j * NN + 16 * cg), v[j]);
          tmem_wait_ld();
#pragma unroll
          for (int cc = 0; cc < 4; ++cc) {
            const int c = 4 * cg + cc;
            if (p < a.npair && c < nbl) {
#pragma unroll
              for (int side = 0; side < 2; ++side) {
                const int y = side ? ys : p;
                if (y < 0) continue;
                const long long at = ((long long)(b0 + c) * a.nring + y) * mstride + m;
                float2 w[MQ];
#pragma unroll
                for (int j = 0; j < MQ; ++j)
                  w[j] = make_float2(__uint_as_float(v[j][4 * cc + 2 * side]), __uint_as_float(v[j][4 * cc + 2 * side + 1]));
                if (nq == MQ && (at % MQ) == 0) {  // whole pieces: 16 or 32 bytes
                  float4* d = reinterpret_cast<float4*>(F + at);
#pragma unroll
                  for (int h = 0; h < MQ / 2; ++h) d[h] = make_float4(w[2 * h].x, w[2 * h].y, w[2 * h + 1].x, w[2 * h + 1].y);
                } else {
                  for (int j = 0; j < nq; ++j) F[at + j] = w[j];
                }
              }
            }
          }
        }
      } else if constexpr (SYN) {
        // north ring p: E + O; its mirror (none for the equator): E - O
        const int p = ptile * 128 + t;
        if (p < a.npair) {
          const int ys = p == a.npair - 1 ? -1 : a.nring - 1 - p;
          float2* F = reinterpret_cast<float2*>(a.out);
          const long long mstride = a.mmax + 1;
#pragma unroll
          for (int c = 0; c < C2N / 2; ++c) {
            if (c < nbl) {
              const float inv = a.lscale / chan_scale(a.bmax, b0 + c, a.sfac);  // a power of two
              const float er = sum[2 * c] * inv, ei = sum[2 * c + 1] * inv;
              const float orr = sum[C2N + 2 * c] * inv, oi = sum[C2N + 2 * c + 1] * inv;
              const long long fb = (long long)(b0 + c) * a.nring;
              F[(fb + p) * mstride + m] = make_float2(er + orr, ei + oi);
              if (ys >= 0) F[(fb + ys) * mstride + m] = make_float2(er - orr, ei - oi);
            }
          }
        }
      } else if (l <= a.lmax) {
        const long long base = alm_base(a.lmax, m);
        // P_l (FP32) times powers of two (mfac, the table and channel scales)
        const float scale = a.coef_pf[base + l] * (m > 0 ? (float)a.mfac : 1.f) * a.lscale;
        float2* out = reinterpret_cast<float2*>(a.out) + (long long)b0 * a.nalm + base + l;
#pragma unroll
        for (int c = 0; c < C2N / 2; ++c)
          if (c < nbl) {  // the channel scale last: exact unless the result itself is subnormal
            const float inv = 1.f / chan_scale(a.bmax, b0 + c, a.sfac);
            out[(long long)c * a.nalm] = make_float2(scale * sum[2 * c] * inv, scale * sum[2 * c + 1] * inv);
          }
      }
    }
    if (*abort_flag != 0 && t == 0) atomicExch(a.status, (int)HPX_ERR_TIMEOUT);
    __syncthreads();
    if (warp == 0)
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kAlloc));
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

// A row-major matrix of `rows` rows of 128 bytes (32 floats or 64 16-bit
// values), read as tiles of box_rows rows in the 128-byte swizzle; rows past
// the end read as zero.
bool encode_rows128(void* out, const void* base, unsigned long long rows, unsigned box_rows, int esize) {
  auto enc = tensor_map_encoder();
  if (!enc) return false;
  const unsigned kw = 128 / esize;
  cuuint64_t dims[2] = {kw, (cuuint64_t)(rows > 0 ? rows : 1)};
  cuuint64_t strides[1] = {128};
  cuuint32_t box[2] = {kw, box_rows}, es[2] = {1, 1};
  return enc(reinterpret_cast<CUtensorMap*>(out),
             esize == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_UINT16, 2,
             const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

TcArgs tc_args(const hpx_plan_s* p, bool syn, float* out, int b0, int nb, double mfac) {
  TcArgs a;
  a.off = syn ? p->d_stab_off : p->d_tab_off;
  a.lstart = syn ? p->d_stab_lstart : p->d_tab_lstart;
  a.ngroup = syn ? p->nptile : p->ngroup;
  a.achunk = p->d_achunk;
  a.coef_pf = p->d_coef_pf;
  a.bmax = p->tc_mode ? p->d_bmax + (syn ? p->bmax_stride : 0) : nullptr;
  a.sfac = syn ? p->tc_sfac_s : p->tc_sfac_a;
  a.lscale = p->tc_mode ? (float)(1.0 / kLamScale) : 1.f;
  a.out = out;
  a.lmax = p->lmax;
  a.mmax = p->mmax;
  a.npair = p->npair;
  a.nring = p->nring;
  a.nalm = p->nalm;
  a.b0 = b0;
  a.nb = nb;
  a.mfac = mfac;
  a.fmt = (uint32_t)p->tc_fmt;
  a.status = p->d_status;
  a.m0 = 0;
  a.nm = p->mmax + 1;
  a.tbase = 0;
  a.ncg = 1;
  a.cg_rows = 0;
  a.withhold = p->test_withhold;
  return a;
}

// One tile launch: the lambda descriptors (resident table or a staging
// buffer), the m range, and the table element at the descriptors' row 0.
struct TileRange {
  const void* tmA;
  const void* tmAlo;
  int m0, nm;
  long long tbase;
};

template <int CP, typename E>
cudaError_t pack_gt_cp(const hpx_plan_s* p, int b0, int nb, bool use_w, cudaStream_t s) {
  static_assert(CP % kPackC == 0, "channel blocks");  // CP >= 8
  const bool x3 = p->tc_mode == 2;
  const size_t smem = (size_t)kPackM * pack_slab(pack_rows(x3)) + kPackC * sizeof(float);
  cudaError_t e = allow_max_smem(k_pack_gt<E>);
  if (e != cudaSuccess) return e;
  E* gt = (E*)p->d_gt + (long long)(b0 / CP) * p->gt_group_elems;  // the group's region
  k_pack_gt<E><<<dim3(p->ngroup, (p->mmax + kPackM) / kPackM, CP / kPackC), 256, smem, s>>>(
      (const float2*)p->d_spec, (const float2*)p->d_etab, p->d_ring, gt, p->npair, p->nring, p->ngroup,
      p->nspec, p->mmax, 4 * CP, b0, nb, use_w ? 1 : 0, x3 ? 1 : 0, p->tc_mode ? p->d_bmax : nullptr, p->tc_sfac_a);
  return cudaGetLastError();
}

template <int CP, typename E>
cudaError_t pack_at_cp(const hpx_plan_s* p, const float* alm, int b0, int nb, double mfac, cudaStream_t s) {
  constexpr int KW = Elt<E>::kw;
  const int nchunk0 = p->lmax / KW + 1;  // chunks of m = 0, the most
  E* at = (E*)p->d_at + (long long)(b0 / CP) * p->at_group_elems;  // the group's region
  k_pack_at<CP, E><<<dim3((nchunk0 + 128 / KW - 1) / (128 / KW), p->mmax + 1), 128, 0, s>>>(
      (const float2*)alm, p->d_coef_pf, p->d_achunk, at, p->lmax, p->mmax, p->nalm, b0, nb, (float)mfac,
      p->tc_mode == 2 ? 1 : 0, p->tc_mode ? p->d_bmax + p->bmax_stride : nullptr, p->tc_sfac_s);
  return cudaGetLastError();
}

template <int CP, bool SYN, int MODE>
cudaError_t tile_cp(const hpx_plan_s* p, float* out, int b0, int nb, double mfac, const TileRange& r,
                    cudaStream_t s) {
  constexpr int NN = 4 * CP;
  cudaError_t e = allow_max_smem(k_legendre_tc<NN, SYN, MODE>);
  if (e != cudaSuccess) return e;
  const CUtensorMap* tmB = reinterpret_cast<const CUtensorMap*>(SYN ? p->tm_at : p->tm_gt);
  constexpr int MQ = tc_mq<NN, SYN, MODE>();
  // all channel groups of [b0, b0 + nb) in one launch, the groups' operand
  // regions (At or Gt) at_group_elems / gt_group_elems apart
  const int ncg = (nb + CP - 1) / CP;
  const dim3 grid((SYN ? p->nptile : (p->lmax + kTcTile) / kTcTile) * ncg, (r.nm + MQ - 1) / MQ);
  TcArgs a = tc_args(p, SYN, out, b0, nb, mfac);
  a.m0 = r.m0;
  a.nm = r.nm;
  a.tbase = r.tbase;
  a.ncg = ncg;
  a.cg_rows = (SYN ? p->at_group_elems : p->gt_group_elems) / (MODE == 0 ? 32 : 64);
  k_legendre_tc<NN, SYN, MODE><<<grid, kTcThreads, TcShape<NN, SYN, MODE>::kSmem, s>>>(
      *reinterpret_cast<const CUtensorMap*>(r.tmA), *reinterpret_cast<const CUtensorMap*>(r.tmAlo), *tmB, a);
  return cudaGetLastError();
}

// Dispatch on the plan's operand type (float for mode 0, else 16-bit).
template <int CP>
cudaError_t pack_gt_t(const hpx_plan_s* p, int b0, int nb, bool use_w, cudaStream_t s) {
  if (p->tc_mode == 0) return pack_gt_cp<CP, float>(p, b0, nb, use_w, s);
  return p->tc_fmt == 1 ? pack_gt_cp<CP, __nv_bfloat16>(p, b0, nb, use_w, s)
                        : pack_gt_cp<CP, __half>(p, b0, nb, use_w, s);
}
template <int CP>
cudaError_t pack_at_t(const hpx_plan_s* p, const float* alm, int b0, int nb, double mfac, cudaStream_t s) {
  if (p->tc_mode == 0) return pack_at_cp<CP, float>(p, alm, b0, nb, mfac, s);
  return p->tc_fmt == 1 ? pack_at_cp<CP, __nv_bfloat16>(p, alm, b0, nb, mfac, s)
                        : pack_at_cp<CP, __half>(p, alm, b0, nb, mfac, s);
}
template <int CP, bool SYN>
cudaError_t tile_t(const hpx_plan_s* p, float* out, int b0, int nb, double mfac, const TileRange& r,
                   cudaStream_t s) {
  switch (p->tc_mode) {
    case 0: if constexpr (CP <= 32) return tile_cp<CP, SYN, 0>(p, out, b0, nb, mfac, r, s); break;
    case 1: return tile_cp<CP, SYN, 1>(p, out, b0, nb, mfac, r, s);  // up to 64 channels either way
    case 2: if constexpr (CP <= 32 || !SYN) return tile_cp<CP, SYN, 2>(p, out, b0, nb, mfac, r, s); break;
  }
  return cudaErrorInvalidValue;
}

template <bool SYN>
cudaError_t tile_nn(const hpx_plan_s* p, float* out, int b0, int nb, double mfac, const TileRange& r,
                    cudaStream_t s) {
  switch (SYN ? p->tc_nn_s : p->tc_nn_a) {
    case 32: return tile_t<8, SYN>(p, out, b0, nb, mfac, r, s);
    case 64: return tile_t<16, SYN>(p, out, b0, nb, mfac, r, s);
    case 128: return tile_t<32, SYN>(p, out, b0, nb, mfac, r, s);
    case 256: return tile_t<64, SYN>(p, out, b0, nb, mfac, r, s);  // (a 64-channel synthesis: mode 1 only)
  }
  return cudaErrorInvalidValue;
}

cudaError_t fill_table(hpx_plan_s* p, bool col, int m0, int nm, long long base, void* hi, void* lo,
                       cudaStream_t s);

// The tile kernel over all m: one launch on the resident table, or one
// launch per m block with the block's slice of the table in a staging
// buffer: copied from the host table (out-of-core plans) or filled by the
// recurrence (streamed plans) on the plan's second stream.  Two staging
// buffers alternate; a copy or fill waits until the launch that last read
// its buffer is done, and a launch waits for its copy or fill, so the next
// block's fill runs beside this block's products.
template <bool SYN>
cudaError_t tile_all(hpx_plan_s* p, float* out, int b0, int nb, double mfac, cudaStream_t s) {
  const bool streamed = (p->flags & HPX_PLAN_LAMBDA_STREAM) != 0;
  if (!p->h_tab && !streamed) {
    const TileRange r{SYN ? p->tm_stab : p->tm_tab, SYN ? p->tm_stablo : p->tm_tablo, 0, p->mmax + 1, 0};
    return tile_nn<SYN>(p, out, b0, nb, mfac, r, s);
  }
  cudaStream_t cs = static_cast<cudaStream_t>(p->copy_stream);
  cudaEvent_t* ev = reinterpret_cast<cudaEvent_t*>(p->stage_events);  // [0, 1] copied, [2, 3] free
  const int nblk = SYN ? p->nblk_col : p->nblk_row;
  const int* bm = SYN ? p->blk_col : p->blk_row;                    // [nblk + 1] m boundaries
  const long long* bb = SYN ? p->blk_col_base : p->blk_row_base;    // [nblk + 1] element boundaries
  const char* hhi = static_cast<const char*>(SYN ? p->h_stab : p->h_tab);
  const char* hlo = static_cast<const char*>(SYN ? p->h_stab_lo : p->h_tab_lo);
  const size_t es = p->tc_mode ? 2 : 4;
  cudaError_t e = cudaSuccess;
  for (int j = 0; j < nblk && e == cudaSuccess; ++j) {
    const int buf = p->stage_next;
    p->stage_next ^= 1;
    const size_t bytes = (size_t)(bb[j + 1] - bb[j]) * es;
    char* d = static_cast<char*>(p->d_stage[buf]);
    e = cudaStreamWaitEvent(cs, ev[2 + buf], 0);
    if (streamed) {
      if (e == cudaSuccess)
        e = fill_table(p, SYN, bm[j], bm[j + 1] - bm[j], bb[j], d, p->tc_mode == 2 ? d + p->stage_bytes : nullptr, cs);
    } else {
      if (e == cudaSuccess) e = cudaMemcpyAsync(d, hhi + (size_t)bb[j] * es, bytes, cudaMemcpyHostToDevice, cs);
      if (e == cudaSuccess && hlo)
        e = cudaMemcpyAsync(d + p->stage_bytes, hlo + (size_t)bb[j] * es, bytes, cudaMemcpyHostToDevice, cs);
    }
    if (e == cudaSuccess) e = cudaEventRecord(ev[buf], cs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev[buf], 0);
    if (e == cudaSuccess) {
      const TileRange r{p->tm_stage[buf], p->tm_stagelo[buf], bm[j], bm[j + 1] - bm[j], bb[j]};
      e = tile_nn<SYN>(p, out, b0, nb, mfac, r, s);
    }
    if (e == cudaSuccess) e = cudaEventRecord(ev[2 + buf], s);
  }
  return e;
}

}  // namespace

int tc_mode_of(int dtype, unsigned flags) {
  switch (dtype) {
    case HPX_F32:
      if (!(flags & HPX_PLAN_TENSOR_CORES)) return -1;
      return (flags & HPX_PLAN_TC_TF32X3) ? 0 : 2;  // FP32 plans: FP16 hi/lo unless 3xTF32 is asked for
    case HPX_F32_BF16: case HPX_F32_FP16: return 1;
    case HPX_F32_BF16X3: case HPX_F32_FP16X3: return 2;
    default: return -1;
  }
}

namespace {

// (the synthesis half of the plan's maxima)
cudaError_t absmax(hpx_plan_s const* p, const float2* x, long long n, long long stride, int b0, int nb,
                   cudaStream_t s) {
  unsigned* bm = p->d_bmax + p->bmax_stride;
  cudaError_t e = cudaMemsetAsync(bm + b0, 0, sizeof(unsigned) * nb, s);
  if (e != cudaSuccess) return e;
  const long long blocks = (n + 1023) / 1024;  // about four values per thread
  k_absmax<<<dim3((unsigned)(blocks < 1024 ? blocks : 1024), nb), 256, 0, s>>>(x, n, stride, b0, bm);
  return cudaGetLastError();
}

}  // namespace

// Channels per synthesis CTA (the tile's N is 4 per channel); a synthesis of
// more channels runs their groups side by side in one launch.
#ifndef HPX_TC_SYN_CHANNELS
#define HPX_TC_SYN_CHANNELS 16
#endif
constexpr int kSynChannels = HPX_TC_SYN_CHANNELS;
// Channels per analysis CTA: 32 for FP32 operands (3xTF32), else this.
#ifndef HPX_TC_ANA_CHANNELS
#define HPX_TC_ANA_CHANNELS 64
#endif
constexpr int kAnaChannels = HPX_TC_ANA_CHANNELS;
static_assert(kAnaChannels == 8 || kAnaChannels == 16 || kAnaChannels == 32 || kAnaChannels == 64, "analysis group");
static_assert(kSynChannels == 8 || kSynChannels == 16 || kSynChannels == 32, "synthesis channel group");
// Channels per synthesis CTA in the single-product modes (partner CTAs of
// a wider transform read each lambda block from L2).
#ifndef HPX_TC_SYN_CHANNELS_FK
#define HPX_TC_SYN_CHANNELS_FK 32
#endif
constexpr int kSynChannelsFK = HPX_TC_SYN_CHANNELS_FK;
static_assert(kSynChannelsFK == 32 || kSynChannelsFK == 64, "single-product synthesis channel group");

int tc_columns(int nbatch, int cap) {
  int cp = 8;
  while (cp < nbatch && cp < cap) cp *= 2;
  return 4 * cp;
}

int tc_channels_per_launch(const hpx_plan_s* p, bool syn) { return (syn ? p->tc_nn_s : p->tc_nn_a) / 4; }

size_t tc_extra_bytes_estimate(int nside, int lmax, int mmax, int nbatch, int mode, bool host_tables) {
  if (mode < 0) return 0;
  const size_t es = mode ? 2 : 4, kw = mode ? 64 : 32, parts = mode == 2 ? 2 : 1;
  const size_t npair = 2 * (size_t)nside, ngroup = (npair + kw - 1) / kw, nptile = (npair + 127) / 128;
  const size_t nna = (size_t)tc_columns(nbatch, mode ? kAnaChannels : 32),
               nns = (size_t)tc_columns(nbatch, mode == 1 ? kSynChannelsFK : kSynChannels);
  size_t chunks = 0, rows = 0;
  for (int m = 0; m <= mmax; ++m) {
    chunks += (size_t)((lmax - m) / kw + 1);
    rows += (size_t)(lmax + 1 - m) + kTcTile;
  }
  const size_t cps = nns / 4, groups = ((size_t)nbatch + cps - 1) / cps;
  const size_t cpa = nna / 4, groups_a = ((size_t)nbatch + cpa - 1) / cpa;
  size_t b = es * (size_t)(mmax + 1) * ngroup * nna * kw * parts * groups_a  // Gt, one region per channel group
             + es * chunks * nns * kw * parts * groups                       // At, likewise
             + (sizeof(int) + sizeof(long long)) * (size_t)(mmax + 1) * (nptile + ngroup) +
             sizeof(long long) * (mmax + 2) + 2 * sizeof(unsigned) * nbatch;
  const size_t col = es * chunks * nptile * 128 * kw, row = es * rows * ngroup * kw;  // upper bounds, a part
  if (host_tables)  // staging buffers at the default size
    return b + 2 * parts * std::min(size_t(1) << 30, (std::max(col, row) + 127) / 128 * 128);
  b += parts * col;           // column table
  if (mode) b += parts * row;  // 16-bit row table
  return b;
}

namespace {

// Exclusive prefix sums of per-entry row counts times the row width; returns the total.
long long offsets_from_rows(std::vector<long long>& v, long long width) {
  long long acc = 0;
  for (auto& x : v) {
    const long long r = x;
    x = acc;
    acc += width * r;
  }
  return acc;
}

// Blocks of consecutive m whose slice of an m-major table (per-m first
// element off[m * per_m], total `total`) fits `cap` elements.  False if one m
// alone exceeds it.
bool make_blocks(const std::vector<long long>& off, int per_m, int mmax, long long total, long long cap,
                 std::vector<int>& bm, std::vector<long long>& bb) {
  bm.assign(1, 0);
  bb.assign(1, 0);
  for (int m = 0; m <= mmax; ++m) {
    const long long end = m < mmax ? off[(size_t)(m + 1) * per_m] : total;
    if (end - bb.back() > cap) {
      if (bm.back() == m) return false;
      bm.push_back(m);
      bb.push_back(off[(size_t)m * per_m]);
      if (end - bb.back() > cap) return false;
    }
  }
  bm.push_back(mmax + 1);
  bb.push_back(total);
  return true;
}

template <typename E>
cudaError_t fill_row_table(hpx_plan_s* p, int m0, int nm, long long base, void* hi, void* lo, cudaStream_t s) {
  constexpr int KW = Elt<E>::kw;
  k_rtab_fill<E><<<dim3((p->ngroup * KW + 127) / 128, nm), 128, 0, s>>>(
      p->d_ring, p->d_coef_cf, p->d_lc, p->d_mu0, p->d_mu1, p->d_tab_lstart, p->d_tab_off, p->lmax, p->npair,
      p->ngroup, m0, base, static_cast<E*>(hi), static_cast<E*>(lo));
  return cudaGetLastError();
}
template <typename E>
cudaError_t fill_col_table(hpx_plan_s* p, int m0, int nm, long long base, void* hi, void* lo, cudaStream_t s) {
  k_ctab_fill<E><<<dim3(p->nptile, nm), 128, 0, s>>>(p->d_ring, p->d_coef_cf, p->d_lc, p->d_mu0, p->d_mu1,
                                                     p->d_stab_lstart, p->d_stab_off, p->lmax, p->npair,
                                                     p->nptile, m0, base, static_cast<E*>(hi), static_cast<E*>(lo));
  return cudaGetLastError();
}
cudaError_t fill_table(hpx_plan_s* p, bool col, int m0, int nm, long long base, void* hi, void* lo,
                       cudaStream_t s) {
  if (p->tc_mode == 0) return col ? fill_col_table<float>(p, m0, nm, base, hi, nullptr, s)
                                  : fill_row_table<float>(p, m0, nm, base, hi, nullptr, s);
  if (p->tc_fmt == 1) return col ? fill_col_table<__nv_bfloat16>(p, m0, nm, base, hi, lo, s)
                                 : fill_row_table<__nv_bfloat16>(p, m0, nm, base, hi, lo, s);
  return col ? fill_col_table<__half>(p, m0, nm, base, hi, lo, s) : fill_row_table<__half>(p, m0, nm, base, hi, lo, s);
}

}  // namespace

void free_tc_host(hpx_plan_s* p) {
  for (void* h : {p->h_tab, p->h_tab_lo, p->h_stab, p->h_stab_lo})
    if (h) cudaFreeHost(h);
  for (void* d : p->d_stage)
    if (d) cudaFree(d);
  delete[] p->blk_row;
  delete[] p->blk_col;
  delete[] p->blk_row_base;
  delete[] p->blk_col_base;
  if (p->stage_events) {
    cudaEvent_t* ev = static_cast<cudaEvent_t*>(p->stage_events);
    for (int i = 0; i < 4; ++i)
      if (ev[i]) cudaEventDestroy(ev[i]);
    delete[] ev;
  }
  if (p->copy_stream) cudaStreamDestroy(static_cast<cudaStream_t>(p->copy_stream));
}

cudaError_t build_tc(hpx_plan_s* p, cudaStream_t s) {
  const int mode = tc_mode_of(p->dtype, p->flags);
  if (mode < 0) return cudaErrorInvalidValue;
  p->tc_mode = mode;
  p->tc_fmt = (p->dtype == HPX_F32_BF16 || p->dtype == HPX_F32_BF16X3) ? 1 : 0;  // FP32 plans: FP16
  const bool host = (p->flags & HPX_PLAN_LAMBDA_HOST) != 0;
  const bool streamed = (p->flags & HPX_PLAN_LAMBDA_STREAM) != 0;
  const int kw = mode ? 64 : 32, es = mode ? 2 : 4, parts = mode == 2 ? 2 : 1;
  // synthesis channels per CTA: kSynChannelsFK for one 16-bit product
  // (accumulated over all K in tensor memory), else kSynChannels
  const int nna = tc_columns(p->nbatch, mode ? kAnaChannels : 32),
            nns = tc_columns(p->nbatch, mode == 1 ? kSynChannelsFK : kSynChannels);
  const int rba = mode == 2 ? 2 * nna : nna, rbs = mode == 2 ? 2 * nns : nns;
  auto dalloc = [&](void** ptr, size_t bytes) -> cudaError_t {
    cudaError_t e = cudaMalloc(ptr, bytes > 0 ? bytes : 16);
    if (e == cudaSuccess) p->bytes += bytes > 0 ? bytes : 16;
    return e;
  };
  cudaError_t e = cudaSuccess;
  // row table layout: built here for the 16-bit types and for out-of-core
  // and streamed plans (the resident FP32 one comes with the CUDA-core table)
  std::vector<long long> roff;
  if (mode || host || streamed) {
    const int ng = (p->npair + kw - 1) / kw;
    p->ngroup = ng;
    const long long nent = (long long)(p->mmax + 1) * ng;
    e = dalloc((void**)&p->d_tab_lstart, sizeof(int) * nent);
    if (e == cudaSuccess) e = dalloc((void**)&p->d_tab_off, sizeof(long long) * nent);
    if (e != cudaSuccess) return e;
    k_rtab_groups<<<dim3((ng + 127) / 128, p->mmax + 1), 128, 0, s>>>(p->d_lc, p->lmax, p->npair, kw, ng,
                                                                       p->d_tab_lstart, p->d_tab_off);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    roff.resize(nent);
    if (e == cudaSuccess) e = cudaMemcpy(roff.data(), p->d_tab_off, sizeof(long long) * nent, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return e;
    p->tab_elems = offsets_from_rows(roff, kw);
    e = cudaMemcpy(p->d_tab_off, roff.data(), sizeof(long long) * nent, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
  }
  // analysis operand, one region per channel group
  p->gt_group_elems = (long long)(p->mmax + 1) * p->ngroup * rba * kw;
  p->gt_groups = (p->nbatch + nna / 4 - 1) / (nna / 4);
  e = dalloc(&p->d_gt, (size_t)es * p->gt_group_elems * p->gt_groups);
  if (e != cudaSuccess) return e;
  // synthesis operand: chunk offsets of each m, then At
  std::vector<long long> ach(p->mmax + 2);
  ach[0] = 0;
  for (int m = 0; m <= p->mmax; ++m) ach[m + 1] = ach[m] + (p->lmax - m) / kw + 1;
  e = dalloc((void**)&p->d_achunk, sizeof(long long) * (p->mmax + 2));
  if (e == cudaSuccess)
    e = cudaMemcpy(p->d_achunk, ach.data(), sizeof(long long) * (p->mmax + 2), cudaMemcpyHostToDevice);
  p->at_group_elems = (long long)ach[p->mmax + 1] * rbs * kw;
  p->at_groups = (p->nbatch + nns / 4 - 1) / (nns / 4);
  if (e == cudaSuccess) e = dalloc(&p->d_at, (size_t)es * p->at_group_elems * p->at_groups);
  p->bmax_stride = p->nbatch;
  if (e == cudaSuccess) e = dalloc((void**)&p->d_bmax, 2 * sizeof(unsigned) * p->nbatch);
  if (e != cudaSuccess) return e;
  // column table layout
  p->nptile = (p->npair + 127) / 128;
  const long long cent = (long long)(p->mmax + 1) * p->nptile;
  e = dalloc((void**)&p->d_stab_lstart, sizeof(int) * cent);
  if (e == cudaSuccess) e = dalloc((void**)&p->d_stab_off, sizeof(long long) * cent);
  if (e != cudaSuccess) return e;
  k_ctab_tiles<<<dim3((p->nptile + 127) / 128, p->mmax + 1), 128, 0, s>>>(p->d_lc, p->lmax, p->npair, kw, p->nptile,
                                                                           p->d_stab_lstart, p->d_stab_off);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  std::vector<long long> coff(cent);
  if (e == cudaSuccess) e = cudaMemcpy(coff.data(), p->d_stab_off, sizeof(long long) * cent, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return e;
  p->stab_elems = offsets_from_rows(coff, 128LL * kw);
  e = cudaMemcpy(p->d_stab_off, coff.data(), sizeof(long long) * cent, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return e;

  if (!host && !streamed) {
    // resident tables
    if (mode) {
      e = dalloc(&p->d_tab, (size_t)es * p->tab_elems);
      if (e == cudaSuccess && mode == 2) e = dalloc(&p->d_tab_lo, (size_t)es * p->tab_elems);
      if (e == cudaSuccess) e = fill_table(p, false, 0, p->mmax + 1, 0, p->d_tab, p->d_tab_lo, s);
      if (e != cudaSuccess) return e;
    }
    e = dalloc(&p->d_stab, (size_t)es * p->stab_elems);
    if (e == cudaSuccess && mode == 2) e = dalloc(&p->d_stab_lo, (size_t)es * p->stab_elems);
    if (e == cudaSuccess) e = fill_table(p, true, 0, p->mmax + 1, 0, p->d_stab, p->d_stab_lo, s);
    if (e != cudaSuccess) return e;
    const void* tablo = p->d_tab_lo ? p->d_tab_lo : p->d_tab;
    const void* stablo = p->d_stab_lo ? p->d_stab_lo : p->d_stab;
    const unsigned long long trows = (unsigned long long)(p->tab_elems / kw);
    const unsigned long long srows = (unsigned long long)(p->stab_elems / kw);
    if (!encode_rows128(p->tm_tab, p->d_tab, trows, kTcTile, es) ||
        !encode_rows128(p->tm_tablo, tablo, trows, kTcTile, es) ||
        !encode_rows128(p->tm_stab, p->d_stab, srows, 128, es) ||
        !encode_rows128(p->tm_stablo, stablo, srows, 128, es)) {
      set_error("cuTensorMapEncodeTiled failed or is unavailable");
      return cudaErrorInvalidValue;
    }
  } else {
    // out-of-core tables: m blocks that fit a staging buffer, filled block by
    // block on the device and copied to pinned host memory; streamed plans:
    // the same blocks, filled anew by every transform
    if (p->stage_bytes == 0) {  // 1 GiB, or less where the larger table part is smaller
      const size_t whole = (size_t)es * (size_t)std::max(p->tab_elems, p->stab_elems);
      p->stage_bytes = std::min(size_t(1) << 30, (whole + 127) / 128 * 128);
    }
    p->stage_bytes = (p->stage_bytes / 128) * 128;
    const long long cap = (long long)(p->stage_bytes / es);
    std::vector<int> rbm, cbm;
    std::vector<long long> rbb, cbb;
    if (!make_blocks(roff, p->ngroup, p->mmax, p->tab_elems, cap, rbm, rbb) ||
        !make_blocks(coff, p->nptile, p->mmax, p->stab_elems, cap, cbm, cbb)) {
      set_error("staging buffers of %zu bytes cannot hold the table slice of a single m", p->stage_bytes);
      return cudaErrorInvalidValue;
    }
    p->nblk_row = (int)rbm.size() - 1;
    p->nblk_col = (int)cbm.size() - 1;
    p->blk_row = new int[rbm.size()];
    p->blk_col = new int[cbm.size()];
    p->blk_row_base = new long long[rbb.size()];
    p->blk_col_base = new long long[cbb.size()];
    std::copy(rbm.begin(), rbm.end(), p->blk_row);
    std::copy(cbm.begin(), cbm.end(), p->blk_col);
    std::copy(rbb.begin(), rbb.end(), p->blk_row_base);
    std::copy(cbb.begin(), cbb.end(), p->blk_col_base);
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) e = dalloc(&p->d_stage[b], p->stage_bytes * parts);
    if (e != cudaSuccess) return e;
    if (host) {
      auto halloc = [&](void** ptr, size_t bytes) -> cudaError_t {
        cudaError_t r = cudaHostAlloc(ptr, bytes > 0 ? bytes : 16, cudaHostAllocDefault);
        if (r == cudaSuccess) p->host_bytes += bytes;
        return r;
      };
      e = halloc(&p->h_tab, (size_t)es * p->tab_elems);
      if (e == cudaSuccess) e = halloc(&p->h_stab, (size_t)es * p->stab_elems);
      if (e == cudaSuccess && mode == 2) e = halloc(&p->h_tab_lo, (size_t)es * p->tab_elems);
      if (e == cudaSuccess && mode == 2) e = halloc(&p->h_stab_lo, (size_t)es * p->stab_elems);
      if (e != cudaSuccess) return e;
      char* shi = static_cast<char*>(p->d_stage[0]);
      char* slo = mode == 2 ? shi + p->stage_bytes : nullptr;
      for (int col = 0; col < 2 && e == cudaSuccess; ++col) {
        const std::vector<int>& bm = col ? cbm : rbm;
        const std::vector<long long>& bb = col ? cbb : rbb;
        char* hhi = static_cast<char*>(col ? p->h_stab : p->h_tab);
        char* hlo = static_cast<char*>(col ? p->h_stab_lo : p->h_tab_lo);
        for (size_t j = 0; j + 1 < bm.size() && e == cudaSuccess; ++j) {
          const size_t bytes = (size_t)(bb[j + 1] - bb[j]) * es;
          e = fill_table(p, col != 0, bm[j], bm[j + 1] - bm[j], bb[j], shi, slo, s);
          if (e == cudaSuccess)
            e = cudaMemcpyAsync(hhi + (size_t)bb[j] * es, shi, bytes, cudaMemcpyDeviceToHost, s);
          if (e == cudaSuccess && slo)
            e = cudaMemcpyAsync(hlo + (size_t)bb[j] * es, slo, bytes, cudaMemcpyDeviceToHost, s);
          if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        }
      }
      if (e != cudaSuccess) return e;
    }
    const unsigned long long srows = (unsigned long long)(p->stage_bytes / 128);
    for (int b = 0; b < 2; ++b) {
      char* base = static_cast<char*>(p->d_stage[b]);
      if (!encode_rows128(p->tm_stage[b], base, srows, 128, es) ||
          !encode_rows128(p->tm_stagelo[b], mode == 2 ? base + p->stage_bytes : base, srows, 128, es)) {
        set_error("cuTensorMapEncodeTiled failed or is unavailable");
        return cudaErrorInvalidValue;
      }
    }
    cudaStream_t cs;
    e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    p->copy_stream = cs;
    cudaEvent_t* ev = new cudaEvent_t[4]();
    p->stage_events = ev;
    for (int i = 0; i < 4 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
  }
  if (!encode_rows128(p->tm_gt, p->d_gt, (unsigned long long)(p->mmax + 1) * p->ngroup * rba * p->gt_groups, nna,
                      es) ||
      !encode_rows128(p->tm_at, p->d_at, (unsigned long long)ach[p->mmax + 1] * rbs * p->at_groups, nns, es)) {
    set_error("cuTensorMapEncodeTiled failed or is unavailable");
    return cudaErrorInvalidValue;
  }
  p->tc_nn_a = nna;
  p->tc_nn_s = nns;
  return cudaSuccess;
}

cudaError_t launch_pack_tc(hpx_plan_s* p, int b0, int nb, bool use_w, cudaStream_t s) {
  // channel scales from the spectra (their largest components were recorded
  // by the ring transform): |S|, |A| <= 2 sqrt(2) w max|component|
  if (p->tc_mode) p->tc_sfac_a = 3.0f * (use_w ? (float)p->w_max : 1.0f);
  switch (p->tc_nn_a) {
    case 32: return pack_gt_t<8>(p, b0, nb, use_w, s);
    case 64: return pack_gt_t<16>(p, b0, nb, use_w, s);
    case 128: return pack_gt_t<32>(p, b0, nb, use_w, s);
    case 256: return pack_gt_t<64>(p, b0, nb, use_w, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_tile_tc(hpx_plan_s* p, float* alm, int b0, int nb, double mfac, cudaStream_t s) {
  return tile_all<false>(p, alm, b0, nb, mfac, s);
}

cudaError_t launch_pack_at_tc(hpx_plan_s* p, const float* alm, int b0, int nb, double mfac, cudaStream_t s) {
  if (p->tc_mode) {  // channel scales from alm: |P_l mfac a| <= 1.2 max(mfac, 1) max|component|
    p->tc_sfac_s = 1.2f * (float)(mfac > 1.0 ? mfac : 1.0);
    cudaError_t e = absmax(p, reinterpret_cast<const float2*>(alm), p->nalm, p->nalm, b0, nb, s);
    if (e != cudaSuccess) return e;
  }
  switch (p->tc_nn_s) {
    case 32: return pack_at_t<8>(p, alm, b0, nb, mfac, s);
    case 64: return pack_at_t<16>(p, alm, b0, nb, mfac, s);
    case 128: return pack_at_t<32>(p, alm, b0, nb, mfac, s);
    case 256: return pack_at_t<64>(p, alm, b0, nb, mfac, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_synthesis_tc(hpx_plan_s* p, int b0, int nb, cudaStream_t s) {
  return tile_all<true>(p, static_cast<float*>(p->d_F), b0, nb, 1.0, s);
}

}  // namespace hpx
