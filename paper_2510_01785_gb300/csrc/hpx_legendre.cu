// Legendre stage of the HEALPix SHT (Sec. III-D Eq. 14-16, Eq. 24-27).
//
// lambda_lm(z) obeys the three-term recurrence of Eq. 16,
//   lambda_l = alpha_l (z lambda_{l-1} - lambda_{l-2} / alpha_{l-1}),
//   alpha_l = sqrt((4 l^2 - 1) / (l^2 - m^2)),
// started from lambda_mm = (-1)^m sqrt(prod_{k<=m} (2k+1)/(2k) / 4 pi) sin^m.
// It is run here in the rescaled variable mu_l = lambda_l / P_l with
// P_m = P_{m+1} = 1 and P_l = (alpha_l / alpha_{l-1}) P_{l-2}, which turns it
// into mu_l = c_l z mu_{l-1} - mu_{l-2} (c_l = alpha_l P_{l-1} / P_l): two
// FP64 operations per step.  P_l does not depend on the ring, so it is
// applied once per output coefficient (analysis) or once per input
// coefficient (synthesis) instead of once per step.
//
// Exponent rescaling: a plan-time pass runs every (m, ring) chain in a
// (mantissa, 2^(-512 k)) representation from lambda_mm until it first
// reaches 2^-200 and records l_c and (mu_{l_c-1}, mu_{l_c}).  Values before
// l_c are below 2^-193 and are dropped; after l_c they stay within the
// double range, so the per-transform kernels run the plain recurrence from
// the recorded state and skip the dropped part of every chain.
//
// Contraction with the rings (analysis) or coefficients (synthesis) uses the
// north/south symmetry lambda_lm(-z) = (-1)^(l+m) lambda_lm(z): each chain
// serves a mirrored ring pair, with S = G(y) + G(y') for even l - m and
// A = G(y) - G(y') for odd l - m.
#include <cooperative_groups.h>

#include <climits>
#include <vector>

#include "hpx_internal.cuh"

namespace cg = cooperative_groups;

namespace hpx {

constexpr int LB = 32;  // l values per block of the recurrence

// ---------------------------------------------------------------------------
// plan-time tables
// ---------------------------------------------------------------------------
// lambda_mm / sin^m theta = (-1)^m sqrt(prod_{k=1..m} (2k+1)/(2k) / (4 pi)),
// the product carried as an unevaluated double-double sum.
__global__ void k_lambda_mm_prefactor(int mmax, double* cmm) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m > mmax) return;
  double hi = 1.0, lo = 0.0;
  for (int k = 1; k <= m; ++k) {
    const double num = 2.0 * k + 1.0, den = 2.0 * k;
    const double qh = num / den;
    const double ql = fma(-qh, den, num) / den;  // num/den = qh + ql
    const double ph = hi * qh;
    double pe = fma(hi, qh, -ph);
    pe = fma(hi, ql, pe);
    pe = fma(lo, qh, pe);
    hi = ph + pe;
    lo = pe - (hi - ph);
  }
  const double inv4pi = 0.079577471545947667884;  // 1 / (4 pi)
  const double r = sqrt(hi * inv4pi) * (1.0 + 0.5 * lo / hi);
  cmm[m] = (m & 1) ? -r : r;
}

// c_l and P_l of the rescaled recurrence for every (l, m); packed like alm.
__global__ void k_recurrence_coefs(int lmax, int mmax, double* coef_c, double* coef_p,
                                   float* coef_pf) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m > mmax) return;
  const long long base = (long long)m * (2 * lmax + 1 - m) / 2;
  coef_c[base + m] = 0.0;
  coef_p[base + m] = 1.0;
  coef_pf[base + m] = 1.0f;
  double p1 = 1.0, p2 = 1.0, a_prev = 0.0;  // P_{l-1}, P_{l-2}, alpha_{l-1}
  const double md = m;
  for (int l = m + 1; l <= lmax; ++l) {
    const double ld = l;
    const double a = sqrt((4.0 * ld * ld - 1.0) / (ld * ld - md * md));
    double P, c;
    if (l == m + 1) {
      P = 1.0;
      c = a;
    } else {
      P = (a / a_prev) * p2;
      c = a * p1 / P;
    }
    coef_c[base + l] = c;
    coef_p[base + l] = P;
    coef_pf[base + l] = (float)P;
    p2 = p1;
    p1 = P;
    a_prev = a;
  }
}

// Start of every chain (m, pair): the first l at which |mu_l| >= 2^-200,
// with (mu_{l-1}, mu_l) there; l_c = lmax + 1 if the chain never gets there.
__global__ void k_chain_scan(const RingInfo* __restrict__ rings, const double* __restrict__ cmm,
                             const double* __restrict__ coef_c, int lmax, int npair, int* lc_tab,
                             double* mu0_tab, double* mu1_tab) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  const int m = blockIdx.y;
  if (p >= npair) return;
  const double z = rings[p].z, s = rings[p].sinth;
  // sin^m by binary powering on (mantissa, exponent) pairs
  int es;
  const double fs = frexp(s, &es);
  double rm = 1.0, bm = fs;
  long long er = 0, eb = 0;
  for (int n = m; n > 0; n >>= 1) {
    int e;
    if (n & 1) {
      rm = frexp(rm * bm, &e);
      er += eb + e;
    }
    if (n > 1) {
      bm = frexp(bm * bm, &e);
      eb = 2 * eb + e;
    }
  }
  int e1;
  const double v0 = frexp(cmm[m] * rm, &e1);
  const long long E = er + (long long)m * es + e1;  // |lambda_mm| in [2^(E-1), 2^E)
  long long k = 0;
  if (E < -(kSigExp - 1)) k = (-(kSigExp - 1) - E + 511) / 512;
  double mu1 = ldexp(v0, (int)(E + 512 * k)), mu2 = 0.0;
  int l = m;
  const long long base = (long long)m * (2 * lmax + 1 - m) / 2;
  while (k > 0 && l < lmax) {
    ++l;
    const double mu = fma(coef_c[base + l] * z, mu1, -mu2);
    mu2 = mu1;
    mu1 = mu;
    if (fabs(mu1) >= 0x1p312) {
      mu1 *= 0x1p-512;
      mu2 *= 0x1p-512;
      --k;
    }
  }
  const long long ci = (long long)m * npair + p;
  if (k > 0) {
    lc_tab[ci] = lmax + 1;
    mu0_tab[ci] = 0.0;
    mu1_tab[ci] = 0.0;
  } else {
    lc_tab[ci] = l;
    mu0_tab[ci] = mu2;
    mu1_tab[ci] = mu1;
  }
}

// ---------------------------------------------------------------------------
// analysis
// ---------------------------------------------------------------------------
// G_m(y) = w_y exp(-i m phi_{0,y}) X_y[m mod N_y], with X_y[N - k] = conj X_y[k]
// (the m-aliasing fold of Eq. 26 for m >= N_y / 2).
template <typename T>
__device__ __forceinline__ C2<T> ring_coef(const C2<T>* __restrict__ spec, const C2<T>* __restrict__ etab,
                                           const RingInfo& R, int m, int b, long long nspec, int use_w) {
  const int N = R.nphi, H = N >> 1;
  const int k = m % N;
  const C2<T>* X = spec + (long long)b * nspec + R.specoff;
  const C2<T> x = (k <= H) ? X[k] : cconj(X[N - k]);
  C2<T> g = cmul(x, etab[R.etab + ((long long)R.sigma * m) % (2LL * N)]);
  if (use_w) g = cscale(g, (T)R.w);
  return g;
}

// Lane tiling of the (LB x 2CP) output block of one warp: each lane owns LPL
// consecutive l and CPL consecutive real components.
template <int C2N> struct LaneTile;
template <> struct LaneTile<2> { static constexpr int CPL = 2, LPL = 1; };
template <> struct LaneTile<4> { static constexpr int CPL = 4, LPL = 1; };
template <> struct LaneTile<8> { static constexpr int CPL = 4, LPL = 2; };
template <> struct LaneTile<16> { static constexpr int CPL = 4, LPL = 4; };
template <> struct LaneTile<32> { static constexpr int CPL = 8, LPL = 4; };

template <typename T> struct MuStride { static constexpr int v = LB + 16 / (int)sizeof(T); };

// S/A coefficients, mu rows (each warp's partial sums of a block reuse its own
// 32 rows once it has read them), the double-buffered block partials, c_l
template <typename T, int CP>
size_t analysis_smem(int nthr) {
  constexpr int C2N = 2 * CP;
  static_assert(LB * C2N <= 32 * MuStride<T>::v, "partials fit a warp's mu rows");
  return sizeof(T) * ((size_t)nthr * 2 * C2N + (size_t)nthr * MuStride<T>::v + 2 * LB * C2N) +
         sizeof(double) * 2 * LB;
}

// The plan-resident lambda table (HPX_PLAN_LAMBDA_TABLE): for every m and
// every group g of 32 consecutive ring pairs, rows l = lstart(m,g)..lmax of 32
// values mu_l (one per pair of the group), lstart = the group's earliest chain
// start; row r of (m, g) at tab[off(m,g) + 32 r].  Written once at plan time
// by the same FP64 recurrence and conversion as the recomputing kernels.
template <typename T> struct LamTab {
  const T* tab;
  const long long* off;
  const int* lstart;
  int ngroup;
};

// One cluster per m, one recurrence chain per thread.  Warps take 32
// consecutive ring pairs (similar start l, so few idle lanes) and are dealt
// round-robin over the cluster's CTAs, so every CTA holds polar and
// equatorial chains alike and none idles at the cluster barrier.  Per block
// of LB l values: the chains write mu into shared memory (from the recurrence,
// or streamed from the lambda table when TAB), each warp contracts its 32
// chains with their S/A ring coefficients, the warps' partial sums are added
// in shared memory, and the cluster adds the CTAs' partials through
// distributed shared memory (double-buffered, one cluster barrier per block).
// Deterministic order.
template <typename T, int CP, bool TAB>
__global__ void __launch_bounds__(512)
k_legendre_analysis(const C2<T>* __restrict__ spec, T* __restrict__ alm, const RingInfo* __restrict__ rings,
                    const C2<T>* __restrict__ etab, const RecCoef<T>* __restrict__ coef_c,
                    const double* __restrict__ coef_p, const int* __restrict__ lc_tab,
                    const double* __restrict__ mu0_tab, const double* __restrict__ mu1_tab, int lmax,
                    int npair, int nring, long long nspec, long long nalm, int b0, int nb, int use_w,
                    const LamTab<T> tb, double mfac) {
  using V = C2<T>;
  constexpr int C2N = 2 * CP;
  constexpr int CPL = LaneTile<C2N>::CPL, LPL = LaneTile<C2N>::LPL, NCQ = C2N / CPL;
  constexpr int MS = MuStride<T>::v;
  cg::cluster_group cluster = cg::this_cluster();
  const int crank = (int)cluster.block_rank(), csize = (int)cluster.num_blocks();
  const int nthr = blockDim.x, nwarp = nthr >> 5;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int m = blockIdx.y;
  const int p = (warp * csize + crank) * 32 + lane;
  const bool active = p < npair;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sG = reinterpret_cast<T*>(smem_raw);      // [nthr][2][C2N]  S, A
  T* sMu = sG + (size_t)nthr * 2 * C2N;        // [nthr][MS]; warp w's [LB][C2N] partials at row 32 w
  T* sC = sMu + (size_t)nthr * MS;             // [2][LB][C2N]
  RecCoef<T>* sCz = reinterpret_cast<RecCoef<T>*>(sC + 2 * LB * C2N);  // [2][LB] c_l of this and the next block

  double z = 0.0, s0 = 0.0, s1 = 0.0;
  int lc = INT_MAX;
  {
    T* g = sG + (size_t)t * 2 * C2N;
    if (active) {
      const int ys = (p == npair - 1) ? -1 : nring - 1 - p;
      const RingInfo Rn = rings[p];
      z = Rn.z;
      const long long ci = (long long)m * npair + p;
      lc = lc_tab[ci];
      s0 = mu0_tab[ci];
      s1 = mu1_tab[ci];
      if (lc > lmax) lc = INT_MAX;
      for (int c = 0; c < CP; ++c) {
        V gn = cmk<V>(0, 0), gs = cmk<V>(0, 0);
        if (c < nb && lc != INT_MAX) {
          gn = ring_coef<T>(spec, etab, Rn, m, b0 + c, nspec, use_w);
          if (ys >= 0) gs = ring_coef<T>(spec, etab, rings[ys], m, b0 + c, nspec, use_w);
        }
        const V S = cadd(gn, gs), A = csub(gn, gs);
        g[2 * c] = S.x;
        g[2 * c + 1] = S.y;
        g[C2N + 2 * c] = A.x;
        g[C2N + 2 * c + 1] = A.y;
      }
    } else {
      for (int c = 0; c < 2 * C2N; ++c) g[c] = (T)0;
    }
  }

  const long long base = alm_base(lmax, m);
  const int lq = lane / NCQ, cq = lane % NCQ;
  const int l0 = lq * LPL, c0 = cq * CPL;
  Recur<T> rc;
  rc.start(z, s0, s1);
  int buf = 0;
  if (t < LB) sCz[t] = (m + t <= lmax) ? coef_c[base + m + t] : RecCoef<T>{};
  // TAB: this warp's group rows (32 coalesced 128-byte rows per block),
  // loaded one block ahead so the loads are in flight during the contraction
  // and the reductions of the block before
  int tls = INT_MAX;
  const T* ttg = nullptr;
  T nxt[TAB ? LB : 1];
  if constexpr (TAB) {
    const int g = warp * csize + crank;
    if (g < tb.ngroup) {
      tls = tb.lstart[(long long)m * tb.ngroup + g];
      ttg = tb.tab + tb.off[(long long)m * tb.ngroup + g] + lane;
    }
#pragma unroll
    for (int i = 0; i < LB; ++i) {
      const int l = m + i;
      nxt[i] = (l >= tls && l <= lmax) ? __ldcs(ttg + (long long)(l - tls) * 32) : (T)0;
    }
  }
  __syncthreads();
  for (int lb0 = m; lb0 <= lmax; lb0 += LB) {
    const RecCoef<T>* cz = sCz + buf * LB;
    // --- recurrence: LB steps of mu_l = c_l z mu_{l-1} - mu_{l-2} ---
    T* myMu = sMu + (size_t)t * MS;
    if constexpr (TAB) {
#pragma unroll
      for (int i4 = 0; i4 < LB; i4 += 4) {
        if constexpr (sizeof(T) == 4) {
          *reinterpret_cast<float4*>(myMu + i4) = make_float4(nxt[i4], nxt[i4 + 1], nxt[i4 + 2], nxt[i4 + 3]);
        } else {
          *reinterpret_cast<double2*>(myMu + i4) = make_double2(nxt[i4], nxt[i4 + 1]);
          *reinterpret_cast<double2*>(myMu + i4 + 2) = make_double2(nxt[i4 + 2], nxt[i4 + 3]);
        }
      }
#pragma unroll
      for (int i = 0; i < LB; ++i) {
        const int l = lb0 + LB + i;
        nxt[i] = (l >= tls && l <= lmax) ? __ldcs(ttg + (long long)(l - tls) * 32) : (T)0;
      }
    } else if (__any_sync(0xffffffffu, lc < lb0 + LB)) {
#pragma unroll
      for (int i4 = 0; i4 < LB; i4 += 4) {
        T v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = rc.step(cz[i4 + u], lb0 + i4 + u, lc);
        if constexpr (sizeof(T) == 4) {
          *reinterpret_cast<float4*>(myMu + i4) = make_float4(v[0], v[1], v[2], v[3]);
        } else {
          *reinterpret_cast<double2*>(myMu + i4) = make_double2(v[0], v[1]);
          *reinterpret_cast<double2*>(myMu + i4 + 2) = make_double2(v[2], v[3]);
        }
      }
    } else {
#pragma unroll
      for (int i = 0; i < LB; ++i) myMu[i] = (T)0;
    }
    const int any_active = __syncthreads_or(lc < lb0 + LB);
    T* cpart = sC + buf * LB * C2N;
    if (any_active) {
      // --- contraction of this warp's 32 chains ---
      T acc[LPL][CPL];
#pragma unroll
      for (int a = 0; a < LPL; ++a)
#pragma unroll
        for (int c = 0; c < CPL; ++c) acc[a][c] = (T)0;
      const T* muw = sMu + (size_t)(warp * 32) * MS + l0;
      const T* gw = sG + (size_t)(warp * 32) * 2 * C2N + c0;
#pragma unroll 4
      for (int j = 0; j < 32; ++j) {
        T mv[LPL], gsv[CPL], gav[CPL];
#pragma unroll
        for (int a = 0; a < LPL; ++a) mv[a] = muw[(size_t)j * MS + a];
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
          gsv[c] = gw[(size_t)j * 2 * C2N + c];
          gav[c] = gw[(size_t)j * 2 * C2N + C2N + c];
        }
#pragma unroll
        for (int a = 0; a < LPL; ++a) {
          const bool odd = ((l0 + a) & 1) != 0;
#pragma unroll
          for (int c = 0; c < CPL; ++c) acc[a][c] = fma(mv[a], odd ? gav[c] : gsv[c], acc[a][c]);
        }
      }
      // this warp's partials over its own mu rows, which only it has read
      T* wp = sMu + (size_t)(warp * 32) * MS;
      __syncwarp();
#pragma unroll
      for (int a = 0; a < LPL; ++a)
#pragma unroll
        for (int c = 0; c < CPL; ++c) wp[(l0 + a) * C2N + c0 + c] = acc[a][c];
      __syncthreads();
      for (int o = t; o < LB * C2N; o += nthr) {
        T s = (T)0;
        for (int w = 0; w < nwarp; ++w) s += sMu[(size_t)(w * 32) * MS + o];
        cpart[o] = s;
      }
    } else {
      for (int o = t; o < LB * C2N; o += nthr) cpart[o] = (T)0;
    }
    // c_l of the next block, into the other half of the double buffer
    if (t < LB) {
      const int l = lb0 + LB + t;
      sCz[(buf ^ 1) * LB + t] = (l <= lmax) ? coef_c[base + l] : RecCoef<T>{};
    }
    // --- cluster reduction; CTA r writes its share of the block ---
    cluster.sync();
    {
      const int nout = LB * C2N;
      const int per = (nout + csize - 1) / csize;
      const int q_end = min(nout, (crank + 1) * per);
      for (int q = crank * per + t; q < q_end; q += nthr) {
        const int part = q & 1, li = (q >> 1) % LB, bb = (q >> 1) / LB;
        const int l = lb0 + li;
        if (l > lmax || bb >= nb) continue;
        const int o = li * C2N + 2 * bb + part;
        T s = (T)0;
        for (int r = 0; r < csize; ++r) s += cluster.map_shared_rank(cpart, r)[o];
        alm[((long long)(b0 + bb) * nalm + base + l) * 2 + part] =
            (T)(coef_p[base + l] * (m > 0 ? mfac : 1.0) * (double)s);
      }
    }
    buf ^= 1;
  }
  cluster.sync();  // peers may still read this CTA's partials
}

// ---------------------------------------------------------------------------
// analysis with the roles split (FP32 plans recomputing lambda)
// ---------------------------------------------------------------------------
// The same sums as k_legendre_analysis, but the first half of the CTA's
// threads (producers, one chain each) only run the FP64 recurrence, writing
// each block of LB values of mu into one of two shared-memory slots, and the
// second half (consumers, consumer i serving producer i's chain) contract the
// blocks, add the warps' and the cluster's partial sums and write alm.  The
// producers do not wait for the sums, so the FP64 pipe is not left idle
// while a CTA contracts and reduces.
//   producer -> consumer: mbarrier full[slot], one arrival per producer,
//     waited with a time limit;
//   among the consumers: named barrier 1;
//   slot reuse and the cluster sums: every thread takes one cluster-barrier
//     phase per block -- consumers once their block's partials are written,
//     producers for block b just before they write block b + 2 into b's
//     slot (the phase that frees it) -- and one more at the end.
// Deterministic order, as the one-role kernel.
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// true once the phase of `bar` with this parity has completed; false after 1 s
__device__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  if (mbar_test(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (unsigned i = 1; i < (1u << 31); ++i) {
    if (mbar_test(bar, parity)) return true;
    if ((i & 63u) == 0 && global_ns() - t0 > 1000000000ull) break;
  }
  return false;
}

template <int CP>
size_t analysis_ws_smem(int nch) {
  constexpr int C2N = 2 * CP;
  return 32 + sizeof(float) * ((size_t)nch * 2 * C2N + 2 * (size_t)nch * MuStride<float>::v + 2 * LB * C2N);
}

template <int CP>
__global__ void __launch_bounds__(1024)
k_legendre_analysis_ws(const float2* __restrict__ spec, float* __restrict__ alm, const RingInfo* __restrict__ rings,
                       const float2* __restrict__ etab, const float2* __restrict__ coef_c,
                       const double* __restrict__ coef_p, const int* __restrict__ lc_tab,
                       const double* __restrict__ mu0_tab, const double* __restrict__ mu1_tab, int lmax,
                       int npair, int nring, long long nspec, long long nalm, int b0, int nb, int use_w,
                       double mfac, int* __restrict__ status) {
  using T = float;
  using V = float2;
  constexpr int C2N = 2 * CP;
  constexpr int CPL = LaneTile<C2N>::CPL, LPL = LaneTile<C2N>::LPL, NCQ = C2N / CPL;
  constexpr int MS = MuStride<T>::v;
  cg::cluster_group cluster = cg::this_cluster();
  const int crank = (int)cluster.block_rank(), csize = (int)cluster.num_blocks();
  const int nch = blockDim.x >> 1;  // chains of the CTA = producer threads = consumer threads
  const int t = threadIdx.x, lane = t & 31;
  const bool producer = t < nch;
  const int ct = producer ? t : t - nch;  // the chain this thread serves
  const int cw = ct >> 5, nw = nch >> 5;  // its warp among its role's warps
  const int m = blockIdx.y;
  const int p = (cw * csize + crank) * 32 + lane;
  const bool active = p < npair;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw);  // [2]
  T* sG = reinterpret_cast<T*>(smem_raw + 32);              // [nch][2][C2N]  S, A
  T* sMu = sG + (size_t)nch * 2 * C2N;                      // [2][nch][MS]; a consumer warp's partials in its rows
  T* sC = sMu + (size_t)2 * nch * MS;                       // [2][LB][C2N]

  double z = 0.0, s0 = 0.0, s1 = 0.0;
  int lc = INT_MAX;
  if (active) {
    const long long ci = (long long)m * npair + p;
    z = rings[p].z;
    lc = lc_tab[ci];
    s0 = mu0_tab[ci];
    s1 = mu1_tab[ci];
    if (lc > lmax) lc = INT_MAX;
  }
  if (producer) {  // the chain's S and A coefficients, as in the one-role kernel
    T* g = sG + (size_t)ct * 2 * C2N;
    if (active) {
      const int ys = (p == npair - 1) ? -1 : nring - 1 - p;
      const RingInfo Rn = rings[p];
      for (int c = 0; c < CP; ++c) {
        V gn = cmk<V>(0, 0), gs = cmk<V>(0, 0);
        if (c < nb && lc != INT_MAX) {
          gn = ring_coef<T>(spec, etab, Rn, m, b0 + c, nspec, use_w);
          if (ys >= 0) gs = ring_coef<T>(spec, etab, rings[ys], m, b0 + c, nspec, use_w);
        }
        const V S = cadd(gn, gs), A = csub(gn, gs);
        g[2 * c] = S.x;
        g[2 * c + 1] = S.y;
        g[C2N + 2 * c] = A.x;
        g[C2N + 2 * c + 1] = A.y;
      }
    } else {
      for (int c = 0; c < 2 * C2N; ++c) g[c] = (T)0;
    }
  }
  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&full[0])), "r"(nch));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&full[1])), "r"(nch));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();  // the last barrier of all the CTA's threads before the roles part

  const long long base = alm_base(lmax, m);
  const int nblk = (lmax - m) / LB + 1;
  if (producer) {
    // ---- the recurrence, block by block into slot b mod 2
    const float2* cl = coef_c + base;
    Recur<float> rc;
    rc.start(z, s0, s1);
    for (int b = 0; b < nblk; ++b) {
      const int lb0 = m + b * LB, slot = b & 1;
      if (b >= 2) cluster.sync();  // phase b - 2: every consumer is done with block b - 2, which used this slot
      T* myMu = sMu + ((size_t)slot * nch + ct) * MS;
      if (__any_sync(0xffffffffu, lc < lb0 + LB)) {
#pragma unroll
        for (int i4 = 0; i4 < LB; i4 += 4) {
          float2 c4[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) c4[u] = (lb0 + i4 + u <= lmax) ? cl[lb0 + i4 + u] : make_float2(0.f, 0.f);
          T v[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) v[u] = rc.step(c4[u], lb0 + i4 + u, lc);
          *reinterpret_cast<float4*>(myMu + i4) = make_float4(v[0], v[1], v[2], v[3]);
        }
      } else {
#pragma unroll
        for (int i = 0; i < LB; i += 4) *reinterpret_cast<float4*>(myMu + i) = make_float4(0.f, 0.f, 0.f, 0.f);
      }
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&full[slot])) : "memory");
    }
    for (int b = nblk > 2 ? nblk - 2 : 0; b < nblk; ++b) cluster.sync();  // the phases of the last blocks
  } else {
    // ---- contraction and sums
    const int lq = lane / NCQ, cq = lane % NCQ;
    const int l0 = lq * LPL, c0 = cq * CPL;
    bool timed_out = false;
    for (int b = 0; b < nblk; ++b) {
      const int lb0 = m + b * LB, slot = b & 1;
      const bool ok = mbar_wait_bounded(&full[slot], (uint32_t)(b >> 1) & 1u);
      if (!ok) timed_out = true;
      T* muS = sMu + (size_t)slot * nch * MS;
      T acc[LPL][CPL];
#pragma unroll
      for (int a = 0; a < LPL; ++a)
#pragma unroll
        for (int c = 0; c < CPL; ++c) acc[a][c] = (T)0;
      if (__all_sync(0xffffffffu, ok) && __any_sync(0xffffffffu, lc < lb0 + LB)) {
        const T* muw = muS + (size_t)(cw * 32) * MS + l0;
        const T* gw = sG + (size_t)(cw * 32) * 2 * C2N + c0;
#pragma unroll 4
        for (int j = 0; j < 32; ++j) {
          T mv[LPL], gsv[CPL], gav[CPL];
#pragma unroll
          for (int a = 0; a < LPL; ++a) mv[a] = muw[(size_t)j * MS + a];
#pragma unroll
          for (int c = 0; c < CPL; ++c) {
            gsv[c] = gw[(size_t)j * 2 * C2N + c];
            gav[c] = gw[(size_t)j * 2 * C2N + C2N + c];
          }
#pragma unroll
          for (int a = 0; a < LPL; ++a) {
            const bool odd = ((l0 + a) & 1) != 0;
#pragma unroll
            for (int c = 0; c < CPL; ++c) acc[a][c] = fma(mv[a], odd ? gav[c] : gsv[c], acc[a][c]);
          }
        }
      }
      // this warp's partials over its own 32 mu rows of the slot, which only it has read
      T* wp = muS + (size_t)(cw * 32) * MS;
      __syncwarp();
#pragma unroll
      for (int a = 0; a < LPL; ++a)
#pragma unroll
        for (int c = 0; c < CPL; ++c) wp[(l0 + a) * C2N + c0 + c] = acc[a][c];
      asm volatile("bar.sync 1, %0;" ::"r"(nch) : "memory");  // the consumers' partials are in
      T* cpart = sC + slot * LB * C2N;
      for (int o = ct; o < LB * C2N; o += nch) {
        T s = (T)0;
        for (int w = 0; w < nw; ++w) s += muS[(size_t)(w * 32) * MS + o];
        cpart[o] = s;
      }
      cluster.sync();  // phase b
      {
        const int nout = LB * C2N;
        const int per = (nout + csize - 1) / csize;
        const int q_end = min(nout, (crank + 1) * per);
        for (int q = crank * per + ct; q < q_end; q += nch) {
          const int part = q & 1, li = (q >> 1) % LB, bb = (q >> 1) / LB;
          const int l = lb0 + li;
          if (l > lmax || bb >= nb) continue;
          const int o = li * C2N + 2 * bb + part;
          T s = (T)0;
          for (int r = 0; r < csize; ++r) s += cluster.map_shared_rank(cpart, r)[o];
          alm[((long long)(b0 + bb) * nalm + base + l) * 2 + part] =
              (T)(coef_p[base + l] * (m > 0 ? mfac : 1.0) * (double)s);
        }
      }
    }
    if (timed_out) atomicExch(status, (int)HPX_ERR_TIMEOUT);
  }
  cluster.sync();  // peers may still read this CTA's partials
}

// ---------------------------------------------------------------------------
// synthesis
// ---------------------------------------------------------------------------
// One thread per chain (m, pair): E_m = sum over even l - m of a_lm lambda_lm,
// O_m = sum over odd l - m; F_m(y) = E + O on the northern ring and
// F_m(y') = E - O on its mirror (Eq. 24 before the ring transform).  The
// block's coefficients (pre-multiplied by P_l) are broadcast from shared
// memory; mu comes from the recurrence, or from the lambda table when TAB.
template <typename T, int CP, bool TAB>
__global__ void __launch_bounds__(128)
k_legendre_synthesis(const T* __restrict__ alm, C2<T>* __restrict__ F, const RingInfo* __restrict__ rings,
                     const RecCoef<T>* __restrict__ coef_c, const float* __restrict__ coef_pf,
                     const double* __restrict__ coef_p, const int* __restrict__ lc_tab,
                     const double* __restrict__ mu0_tab, const double* __restrict__ mu1_tab, int lmax,
                     int mmax, int npair, int nring, long long nalm, int b0, int nb, const LamTab<T> tb,
                     double mfac) {
  using V = C2<T>;
  constexpr int C2N = 2 * CP;
  __shared__ __align__(16) T sA[LB][C2N];
  __shared__ RecCoef<T> sCz[LB];
  __shared__ int sMinLc;
  const int m = blockIdx.y, t = threadIdx.x, nthr = blockDim.x;
  const int p = blockIdx.x * nthr + t;
  const bool active = p < npair;
  double z = 0.0, s0 = 0.0, s1 = 0.0;
  int lc = INT_MAX;
  if (active) {
    z = rings[p].z;
    const long long ci = (long long)m * npair + p;
    lc = lc_tab[ci];
    s0 = mu0_tab[ci];
    s1 = mu1_tab[ci];
    if (lc > lmax) lc = INT_MAX;
  }
  if (t == 0) sMinLc = INT_MAX;
  __syncthreads();
  atomicMin(&sMinLc, lc);
  __syncthreads();
  const int lstart = sMinLc;
  T accE[C2N], accO[C2N];
#pragma unroll
  for (int c = 0; c < C2N; ++c) accE[c] = accO[c] = (T)0;
  const long long base = alm_base(lmax, m);
  Recur<T> rc;
  rc.start(z, s0, s1);
  if (lstart <= lmax) {
    for (int lb0 = m + ((lstart - m) / LB) * LB; lb0 <= lmax; lb0 += LB) {
      for (int q = t; q < LB * C2N; q += nthr) {
        const int li = q / C2N, c = q % C2N, bb = c >> 1, part = c & 1;
        const int l = lb0 + li;
        T v = (T)0;
        if (l <= lmax && bb < nb && !(m == 0 && part == 1)) {
          const T a = alm[((long long)(b0 + bb) * nalm + base + l) * 2 + part];
          if constexpr (sizeof(T) == 4) v = coef_pf[base + l] * (m > 0 ? (float)mfac : 1.0f) * a;
          else v = (T)(coef_p[base + l] * (m > 0 ? mfac : 1.0) * (double)a);
        }
        sA[li][c] = v;
      }
      if (t < LB) sCz[t] = (lb0 + t <= lmax) ? coef_c[base + lb0 + t] : RecCoef<T>{};
      __syncthreads();
      // a warp whose chains all start after this block has nothing to add
      if (TAB && __any_sync(0xffffffffu, lc < lb0 + LB)) {
        const int g = p >> 5;
        const bool gok = g < tb.ngroup;
        const int ls = gok ? tb.lstart[(long long)m * tb.ngroup + g] : INT_MAX;
        const T* tg = tb.tab + (gok ? tb.off[(long long)m * tb.ngroup + g] : 0) + (p & 31);
#pragma unroll
        for (int h = 0; h < LB; h += 16) {
          T mv[16];
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const int l = lb0 + h + i;
            mv[i] = (l >= ls && l <= lmax) ? __ldcs(tg + (long long)(l - ls) * 32) : (T)0;
          }
#pragma unroll
          for (int i = 0; i < 16; i += 2) {
#pragma unroll
            for (int c = 0; c < C2N; ++c) accE[c] = fma(mv[i], sA[h + i][c], accE[c]);
#pragma unroll
            for (int c = 0; c < C2N; ++c) accO[c] = fma(mv[i + 1], sA[h + i + 1][c], accO[c]);
          }
        }
      } else if (!TAB && __any_sync(0xffffffffu, lc < lb0 + LB)) {
#pragma unroll 4
        for (int i = 0; i < LB; i += 2) {
          {
            const T mf = rc.step(sCz[i], lb0 + i, lc);
#pragma unroll
            for (int c = 0; c < C2N; ++c) accE[c] = fma(mf, sA[i][c], accE[c]);
          }
          {
            const T mf = rc.step(sCz[i + 1], lb0 + i + 1, lc);
#pragma unroll
            for (int c = 0; c < C2N; ++c) accO[c] = fma(mf, sA[i + 1][c], accO[c]);
          }
        }
      }
      __syncthreads();
    }
  }
  if (active) {
    const int ys = (p == npair - 1) ? -1 : nring - 1 - p;
#pragma unroll
    for (int bb = 0; bb < CP; ++bb) {
      if (bb < nb) {
        const V e = cmk<V>(accE[2 * bb], accE[2 * bb + 1]);
        const V o = cmk<V>(accO[2 * bb], accO[2 * bb + 1]);
        F[((long long)(b0 + bb) * nring + p) * (mmax + 1) + m] = cadd(e, o);
        if (ys >= 0) F[((long long)(b0 + bb) * nring + ys) * (mmax + 1) + m] = csub(e, o);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static void analysis_shape(int npair, int* nthr, int* csize) {
  if (npair <= 256) {
    *nthr = ((npair + 31) / 32) * 32;
    *csize = 1;
  } else {
    *nthr = npair / 8 > 256 ? npair / 8 : 256;
    *csize = (npair + *nthr - 1) / *nthr;
  }
}

template <typename T>
static LamTab<T> lam_tab(const hpx_plan_s* p) {
  LamTab<T> tb;
  tb.tab = static_cast<const T*>(p->d_tab);
  tb.off = p->d_tab_off;
  tb.lstart = p->d_tab_lstart;
  tb.ngroup = p->ngroup;
  return tb;
}

template <typename T, int CP, bool TAB>
static cudaError_t launch_analysis_cp(const hpx_plan_s* p, T* alm, bool use_w, double mfac, cudaStream_t s,
                                      int* nlaunch) {
  using V = C2<T>;
  int nthr, csize;
  analysis_shape(p->npair, &nthr, &csize);
  const size_t smem = analysis_smem<T, CP>(nthr);
  cudaError_t e = allow_max_smem(k_legendre_analysis<T, CP, TAB>);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(csize, p->mmax + 1, 1);
  cfg.blockDim = dim3(nthr, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = csize;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  for (int b0 = 0; b0 < p->nbatch; b0 += CP) {
    const int nb = (p->nbatch - b0) < CP ? (p->nbatch - b0) : CP;
    e = cudaLaunchKernelEx(&cfg, k_legendre_analysis<T, CP, TAB>, (const V*)p->d_spec, alm,
                           (const RingInfo*)p->d_ring, (const V*)p->d_etab, rec_coefs<T>(p),
                           (const double*)p->d_coef_p, (const int*)p->d_lc, (const double*)p->d_mu0,
                           (const double*)p->d_mu1, p->lmax, p->npair, p->nring, p->nspec, p->nalm, b0, nb,
                           use_w ? 1 : 0, lam_tab<T>(p), mfac);
    if (e != cudaSuccess) return e;
    ++*nlaunch;
  }
  return cudaGetLastError();
}

template <typename T, int CP>
static cudaError_t launch_analysis_sel(const hpx_plan_s* p, T* alm, bool use_w, double mfac, cudaStream_t s,
                                       int* nlaunch) {
  return p->d_tab ? launch_analysis_cp<T, CP, true>(p, alm, use_w, mfac, s, nlaunch)
                  : launch_analysis_cp<T, CP, false>(p, alm, use_w, mfac, s, nlaunch);
}

template <typename T>
static int pick_cp(const hpx_plan_s* p) {
  int nthr, csize;
  analysis_shape(p->npair, &nthr, &csize);
  const int cmax = sizeof(T) == 4 ? 16 : 8;
  int cp = 1;
  while (cp < p->nbatch && cp < cmax) cp *= 2;
  auto fits = [&](int c) {
    size_t sm = 0;
    switch (c) {
      case 1: sm = analysis_smem<T, 1>(nthr); break;
      case 2: sm = analysis_smem<T, 2>(nthr); break;
      case 4: sm = analysis_smem<T, 4>(nthr); break;
      case 8: sm = analysis_smem<T, 8>(nthr); break;
      default: sm = analysis_smem<T, 16>(nthr); break;
    }
    return sm <= 200 * 1024;
  };
  while (cp > 1 && !fits(cp)) cp /= 2;
  return cp;
}

// The split-role analysis (FP32, lambda recomputed): clusters as for the
// one-role kernel, twice the threads (producers and consumers).
template <int CP>
static cudaError_t launch_analysis_ws_cp(const hpx_plan_s* p, float* alm, bool use_w, double mfac, cudaStream_t s,
                                         int* nlaunch) {
  int nthr, csize;
  analysis_shape(p->npair, &nthr, &csize);
  const size_t smem = analysis_ws_smem<CP>(nthr);
  cudaError_t e = allow_max_smem(k_legendre_analysis_ws<CP>);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(csize, p->mmax + 1, 1);
  cfg.blockDim = dim3(2 * nthr, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = csize;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  for (int b0 = 0; b0 < p->nbatch; b0 += CP) {
    const int nb = (p->nbatch - b0) < CP ? (p->nbatch - b0) : CP;
    e = cudaLaunchKernelEx(&cfg, k_legendre_analysis_ws<CP>, (const float2*)p->d_spec, alm,
                           (const RingInfo*)p->d_ring, (const float2*)p->d_etab, (const float2*)p->d_coef_cf,
                           (const double*)p->d_coef_p, (const int*)p->d_lc, (const double*)p->d_mu0,
                           (const double*)p->d_mu1, p->lmax, p->npair, p->nring, p->nspec, p->nalm, b0, nb,
                           use_w ? 1 : 0, mfac, p->d_status);
    if (e != cudaSuccess) return e;
    ++*nlaunch;
  }
  return cudaGetLastError();
}

// Channels per launch of the split-role analysis: the largest power of two
// up to cap with which two CTAs fit an SM (0 if none).  With one CTA per SM
// (512 chains per CTA at Nside 2048, or wide channel groups) every cluster
// barrier idles the SM's FP64 pipe, and the one-role kernel, whose CTAs
// share SMs with other clusters', is faster (252 against 295 ms at Nside
// 2048 / lmax 6143 / 4 channels).
static int pick_cp_ws(int npair, int cap) {
  int nthr, csize;
  analysis_shape(npair, &nthr, &csize);
  if (nthr > 256) return 0;
  for (int cp = cap; cp >= 1; cp /= 2) {
    size_t sm = 0;
    switch (cp) {
      case 1: sm = analysis_ws_smem<1>(nthr); break;
      case 2: sm = analysis_ws_smem<2>(nthr); break;
      case 4: sm = analysis_ws_smem<4>(nthr); break;
      case 8: sm = analysis_ws_smem<8>(nthr); break;
      default: sm = analysis_ws_smem<16>(nthr); break;
    }
    if (sm <= 112 * 1024) return cp;
  }
  return 0;
}

template <typename T>
cudaError_t launch_analysis(const hpx_plan_s* p, T* alm, bool use_w, double mfac, cudaStream_t s, int* nlaunch) {
  if constexpr (sizeof(T) == 4) {
    // FP32 recomputing lambda: the split-role kernel, unless its channel
    // groups would need more launches (each reruns the recurrence)
    if (!p->d_tab) {
      const int cp_one = pick_cp<T>(p), cp_ws = pick_cp_ws(p->npair, cp_one);
      if (cp_ws > 0 && (p->nbatch + cp_ws - 1) / cp_ws == (p->nbatch + cp_one - 1) / cp_one) {
        switch (cp_ws) {
          case 1: return launch_analysis_ws_cp<1>(p, alm, use_w, mfac, s, nlaunch);
          case 2: return launch_analysis_ws_cp<2>(p, alm, use_w, mfac, s, nlaunch);
          case 4: return launch_analysis_ws_cp<4>(p, alm, use_w, mfac, s, nlaunch);
          case 8: return launch_analysis_ws_cp<8>(p, alm, use_w, mfac, s, nlaunch);
          default: return launch_analysis_ws_cp<16>(p, alm, use_w, mfac, s, nlaunch);
        }
      }
    }
  }
  switch (pick_cp<T>(p)) {
    case 1: return launch_analysis_sel<T, 1>(p, alm, use_w, mfac, s, nlaunch);
    case 2: return launch_analysis_sel<T, 2>(p, alm, use_w, mfac, s, nlaunch);
    case 4: return launch_analysis_sel<T, 4>(p, alm, use_w, mfac, s, nlaunch);
    case 8: return launch_analysis_sel<T, 8>(p, alm, use_w, mfac, s, nlaunch);
    default:
      if constexpr (sizeof(T) == 4) return launch_analysis_sel<T, 16>(p, alm, use_w, mfac, s, nlaunch);
      else return launch_analysis_sel<T, 8>(p, alm, use_w, mfac, s, nlaunch);
  }
}

template <typename T, int CP, bool TAB>
static cudaError_t launch_synthesis_cp(const hpx_plan_s* p, const T* alm, double mfac, cudaStream_t s,
                                       int* nlaunch) {
  using V = C2<T>;
  const int nthr = 128;
  dim3 grid((p->npair + nthr - 1) / nthr, p->mmax + 1);
  for (int b0 = 0; b0 < p->nbatch; b0 += CP) {
    const int nb = (p->nbatch - b0) < CP ? (p->nbatch - b0) : CP;
    k_legendre_synthesis<T, CP, TAB><<<grid, nthr, 0, s>>>(
        alm, (V*)p->d_F, p->d_ring, rec_coefs<T>(p), p->d_coef_pf, p->d_coef_p, p->d_lc, p->d_mu0, p->d_mu1,
        p->lmax, p->mmax, p->npair, p->nring, p->nalm, b0, nb, lam_tab<T>(p), mfac);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    ++*nlaunch;
  }
  return cudaSuccess;
}

template <typename T, int CP>
static cudaError_t launch_synthesis_sel(const hpx_plan_s* p, const T* alm, double mfac, cudaStream_t s,
                                        int* nlaunch) {
  return p->d_tab ? launch_synthesis_cp<T, CP, true>(p, alm, mfac, s, nlaunch)
                  : launch_synthesis_cp<T, CP, false>(p, alm, mfac, s, nlaunch);
}

template <typename T>
cudaError_t launch_synthesis(const hpx_plan_s* p, const T* alm, double mfac, cudaStream_t s, int* nlaunch) {
  int cp = 1;
  const int cmax = sizeof(T) == 4 ? 16 : 8;
  while (cp < p->nbatch && cp < cmax) cp *= 2;
  switch (cp) {
    case 1: return launch_synthesis_sel<T, 1>(p, alm, mfac, s, nlaunch);
    case 2: return launch_synthesis_sel<T, 2>(p, alm, mfac, s, nlaunch);
    case 4: return launch_synthesis_sel<T, 4>(p, alm, mfac, s, nlaunch);
    case 8: return launch_synthesis_sel<T, 8>(p, alm, mfac, s, nlaunch);
    default:
      if constexpr (sizeof(T) == 4) return launch_synthesis_sel<T, 16>(p, alm, mfac, s, nlaunch);
      else return launch_synthesis_sel<T, 8>(p, alm, mfac, s, nlaunch);
  }
}

// c_l as the double-FP32 pairs of the FP32 plans' recurrence
__global__ void k_coef_pairs(const double* __restrict__ coef_c, float2* __restrict__ coef_cf, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const Df d = df_of(coef_c[i]);
    coef_cf[i] = make_float2(d.hi, d.lo);
  }
}

cudaError_t build_recurrence_tables(hpx_plan_s* p, cudaStream_t s) {
  const int mb = (p->mmax + 1 + 127) / 128;
  k_lambda_mm_prefactor<<<mb, 128, 0, s>>>(p->mmax, p->d_cmm);
  k_recurrence_coefs<<<mb, 128, 0, s>>>(p->lmax, p->mmax, p->d_coef_c, p->d_coef_p, p->d_coef_pf);
  const long long nb = (p->nalm + 255) / 256;
  k_coef_pairs<<<(unsigned)(nb < 4096 ? nb : 4096), 256, 0, s>>>(p->d_coef_c, p->d_coef_cf, p->nalm);
  k_chain_scan<<<dim3((p->npair + 127) / 128, p->mmax + 1), 128, 0, s>>>(
      p->d_ring, p->d_cmm, p->d_coef_c, p->lmax, p->npair, p->d_lc, p->d_mu0, p->d_mu1);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// plan-resident lambda table
// ---------------------------------------------------------------------------
// Earliest chain start of each (m, 32-pair group) and its number of rows.
__global__ void k_table_groups(const int* __restrict__ lc_tab, int lmax, int npair, int ngroup, int align,
                               int* lstart, long long* rows) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  const int m = blockIdx.y;
  if (g >= ngroup) return;
  int ls = lmax + 1;
  for (int j = 0; j < 32; ++j) {
    const int p = g * 32 + j;
    if (p < npair) ls = min(ls, lc_tab[(long long)m * npair + p]);
  }
  // for the tensor-core analysis: aligned down to its tile grid m + align j,
  // so that a group covers a tile either entirely or not at all (the extra
  // rows hold zeros)
  if (ls <= lmax) ls = m + ((ls - m) / align) * align;
  lstart[(long long)m * ngroup + g] = ls;
  rows[(long long)m * ngroup + g] = lmax + 1 - ls;
}

// Rows of every group: the recurrence of the per-transform kernels (same
// operations, same conversion), zero before a chain's start and for the
// padding lanes of a group.
template <typename T>
__global__ void k_table_fill(const RingInfo* __restrict__ rings, const RecCoef<T>* __restrict__ coef_c,
                             const int* __restrict__ lc_tab, const double* __restrict__ mu0_tab,
                             const double* __restrict__ mu1_tab, const int* __restrict__ lstart,
                             const long long* __restrict__ off, int lmax, int npair, int ngroup, T* tab) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  const int m = blockIdx.y;
  const int g = p >> 5;
  if (g >= ngroup) return;
  const int ls = lstart[(long long)m * ngroup + g];
  T* out = tab + off[(long long)m * ngroup + g] + (p & 31);
  if (p >= npair) {
    for (int l = ls; l <= lmax; ++l) out[(long long)(l - ls) * 32] = (T)0;
    return;
  }
  const long long ci = (long long)m * npair + p;
  const int lc = lc_tab[ci];
  Recur<T> rc;
  rc.start(rings[p].z, mu0_tab[ci], mu1_tab[ci]);
  const long long base = alm_base(lmax, m);
  for (int l = ls; l <= lmax; ++l) out[(long long)(l - ls) * 32] = rc.step(coef_c[base + l], l, lc);
}

template <typename T>
cudaError_t build_lambda_table(hpx_plan_s* p, cudaStream_t s) {
  const int ng = (p->npair + 31) / 32;
  p->ngroup = ng;
  const long long nent = (long long)(p->mmax + 1) * ng;
  cudaError_t e = cudaMalloc((void**)&p->d_tab_lstart, sizeof(int) * nent);
  if (e != cudaSuccess) return e;
  p->bytes += sizeof(int) * nent;
  e = cudaMalloc((void**)&p->d_tab_off, sizeof(long long) * nent);
  if (e != cudaSuccess) return e;
  p->bytes += sizeof(long long) * nent;
  k_table_groups<<<dim3((ng + 127) / 128, p->mmax + 1), 128, 0, s>>>(
      p->d_lc, p->lmax, p->npair, ng, (p->flags & HPX_PLAN_TENSOR_CORES) ? kTcTile : 1, p->d_tab_lstart, p->d_tab_off);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return e;
  std::vector<long long> rows(nent);
  e = cudaMemcpy(rows.data(), p->d_tab_off, sizeof(long long) * nent, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return e;
  long long acc = 0;
  for (long long i = 0; i < nent; ++i) {
    const long long r = rows[i];
    rows[i] = acc;
    acc += 32 * r;
  }
  p->tab_elems = acc;
  e = cudaMemcpy(p->d_tab_off, rows.data(), sizeof(long long) * nent, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return e;
  e = cudaMalloc(&p->d_tab, sizeof(T) * (acc > 0 ? acc : 1));
  if (e != cudaSuccess) return e;
  p->bytes += sizeof(T) * (acc > 0 ? acc : 1);
  k_table_fill<T><<<dim3((ng * 32 + 127) / 128, p->mmax + 1), 128, 0, s>>>(
      p->d_ring, rec_coefs<T>(p), p->d_lc, p->d_mu0, p->d_mu1, p->d_tab_lstart, p->d_tab_off, p->lmax, p->npair,
      ng, static_cast<T*>(p->d_tab));
  return cudaGetLastError();
}

template cudaError_t build_lambda_table<float>(hpx_plan_s*, cudaStream_t);
template cudaError_t build_lambda_table<double>(hpx_plan_s*, cudaStream_t);
template cudaError_t launch_analysis<float>(const hpx_plan_s*, float*, bool, double, cudaStream_t, int*);
template cudaError_t launch_analysis<double>(const hpx_plan_s*, double*, bool, double, cudaStream_t, int*);
template cudaError_t launch_synthesis<float>(const hpx_plan_s*, const float*, double, cudaStream_t, int*);
template cudaError_t launch_synthesis<double>(const hpx_plan_s*, const double*, double, cudaStream_t, int*);

}  // namespace hpx
