// Ring Fourier stage of the HEALPix SHT (Sec. III-D Eq. 13, Sec. III-E).
//
// Every ring y holds N_y = 4i (polar caps) or 4 nside (equatorial belt)
// equally spaced pixels.  A real ring of length N is transformed through a
// complex transform of half length H = N/2 (even samples as real parts, odd
// samples as imaginary parts).  When H is a power of two that transform is a
// power-of-two FFT in shared memory; otherwise it is Bluestein's chirp-z
// transform (Eq. 17-23): chirp multiply, a power-of-two circular convolution
// done as FFT -> pointwise product with the precomputed kernel spectrum ->
// inverse FFT, and a final chirp multiply.  One CTA handles one (ring,
// channel); the whole transform stays in shared memory, so each stage reads
// its input from HBM once and writes its output once.  Belt rings (all of
// length 4 nside) and cap rings are launched separately, each launch with the
// shared memory its longest transform needs; from Nside 512 the cap rings are
// three launches by transform length and the belt launch runs on a second
// stream beside them (see ring_launches); a ring's channels are adjacent
// CTAs, so its chirp and kernel spectrum are read from HBM once.  Bluestein's
// convolution input is zero in its upper half and only its lower half of
// outputs is used, so the first forward pass and the last inverse pass are
// pruned to those halves.
//
// The power-of-two FFT is a Stockham (self-sorting) transform: radix-16
// passes, then one radix-8, -4 or -2 pass if log2 M is not a multiple of 4,
// natural order in and out.  Each pass reads its butterflies' inputs into
// registers, synchronises, and writes the outputs.  Shared-memory element i
// lives at i + i / 16 (one unused slot after every 16): the pass reads
// j + r M/R and writes (j - k) R + k + r Ns, with the thread index j
// contiguous across a warp, so every access of a half-warp falls on distinct
// bank pairs, and for every stride a multiple of 16 the R addresses of a
// thread are one base plus multiples of one stride (no per-element index
// arithmetic: the kernels are bound by instruction issue, and this layout
// took the ring transforms from 0.73 / 1.52 to 0.52 / 0.88 ms at Nside 1024,
// 8 FP32 channels, against a row-wise XOR swizzle).  One twiddle per
// butterfly comes from the table; its powers are formed by multiplication,
// at most four deep.
//
// Chirp and phase angles pi r / N are reduced exactly in integers before the
// FP64 sincospi that fills the tables.
#include "hpx_internal.cuh"

namespace hpx {

__device__ __forceinline__ int brev(int k, int logm) {
  return (int)(__brev((unsigned)k) >> (32 - logm));
}

// shared-memory position of FFT element i: one unused element after every
// 16, so that element i + 16 t sits t bank pairs further on
__device__ __forceinline__ int spos(int i) { return i + (i >> 4); }
__host__ __device__ inline size_t padded_len(size_t n) { return n + (n >> 4) + 1; }  // the c2r fold writes element n

// Radix-2 decimation in frequency (natural order in, bit-reversed order out),
// used once per plan to transform the Bluestein kernels in FP64.
template <typename V>
__device__ void fft_dif(V* buf, int logm, const V* __restrict__ tw, int logtw, bool inv) {
  const int half_n = 1 << (logm - 1);
  for (int s = logm - 1; s >= 0; --s) {
    const int half = 1 << s;
    for (int t = threadIdx.x; t < half_n; t += blockDim.x) {
      const int pos = t & (half - 1);
      const int i0 = ((t >> s) << (s + 1)) + pos;
      const int i1 = i0 + half;
      V w = tw[pos << (logtw - s - 1)];
      if (inv) w.y = -w.y;
      const V a = buf[i0], b = buf[i1];
      buf[i0] = cadd(a, b);
      buf[i1] = cmul(csub(a, b), w);
    }
    __syncthreads();
  }
}

// x * (-i) (forward) or x * (+i) (inverse)
template <bool INV, typename V> __device__ __forceinline__ V rot90(V x) {
  return INV ? cmk<V>(-x.y, x.x) : cmk<V>(x.y, -x.x);
}

// In-register DFT of length R in {2, 4, 8, 16} (8: decimation in frequency
// down to length 2; 16: two levels of length 4), sign -1 (forward) or +1
// (INV).  Natural order in and out.  For R = 16, NZ = 8 says inputs 8..15
// are zero and NO = 8 that only outputs 0..7 are wanted (the others are then
// left unset).
template <int R, bool INV, int NZ = R, int NO = R, typename V>
__device__ __forceinline__ void dft_small(V (&v)[R]) {
  static_assert((NZ == R && NO == R) || R == 16, "pruning is for radix 16");
  using T = decltype(V::x);
  if constexpr (R == 2) {
    const V a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  } else if constexpr (R == 4) {
    const V u0 = cadd(v[0], v[2]), u1 = cadd(v[1], v[3]);
    const V w0 = csub(v[0], v[2]), w1 = rot90<INV>(csub(v[1], v[3]));
    v[0] = cadd(u0, u1);
    v[2] = csub(u0, u1);
    v[1] = cadd(w0, w1);
    v[3] = csub(w0, w1);
  } else if constexpr (R == 16) {
    // 16 = 4 x 4: DFT4 over n1 of x[4 n1 + n2], times W16^(n2 k1), DFT4
    // over n2; output k1 + 4 k2
    const T h = (T)0.70710678118654752440, c1 = (T)0.92387953251128675613, s1 = (T)0.38268343236508977173;
    V y[4][4];
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) {
      if constexpr (NZ == 8) {  // inputs 4 n1 + n2 with n1 >= 2 are zero
        const V a = v[n2], b = v[4 + n2], rb = rot90<INV>(b);
        y[n2][0] = cadd(a, b);
        y[n2][1] = cadd(a, rb);
        y[n2][2] = csub(a, b);
        y[n2][3] = csub(a, rb);
      } else {
#pragma unroll
        for (int n1 = 0; n1 < 4; ++n1) y[n2][n1] = v[4 * n1 + n2];
        dft_small<4, INV>(y[n2]);
      }
    }
    // W16^e = (cos, -+sin)(pi e / 8) for e = n2 k1 in {1, 2, 3, 4, 6, 9}
    auto tw16 = [&](V x, T c, T s) { return INV ? cmk<V>(x.x * c - x.y * s, x.x * s + x.y * c)
                                               : cmk<V>(x.x * c + x.y * s, x.y * c - x.x * s); };
    y[1][1] = tw16(y[1][1], c1, s1);
    y[1][2] = tw16(y[1][2], h, h);
    y[1][3] = tw16(y[1][3], s1, c1);
    y[2][1] = tw16(y[2][1], h, h);
    y[2][2] = rot90<INV>(y[2][2]);
    y[2][3] = tw16(y[2][3], -h, h);
    y[3][1] = tw16(y[3][1], s1, c1);
    y[3][2] = tw16(y[3][2], -h, h);
    y[3][3] = tw16(y[3][3], -c1, -s1);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
      V z[4] = {y[0][k1], y[1][k1], y[2][k1], y[3][k1]};
      if constexpr (NO == 8) {  // outputs k1 + 4 k2 with k2 < 2 only
        const V u0 = cadd(z[0], z[2]), u1 = cadd(z[1], z[3]);
        const V w0 = csub(z[0], z[2]), w1 = rot90<INV>(csub(z[1], z[3]));
        v[k1] = cadd(u0, u1);
        v[k1 + 4] = cadd(w0, w1);
      } else {
        dft_small<4, INV>(z);
#pragma unroll
        for (int k2 = 0; k2 < 4; ++k2) v[k1 + 4 * k2] = z[k2];
      }
    }
  } else {
    const T h = (T)0.70710678118654752440;  // 1/sqrt(2)
    V u[4], w[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      u[r] = cadd(v[r], v[r + 4]);
      w[r] = csub(v[r], v[r + 4]);
    }
    // w[r] *= exp(-+ 2 pi i r / 8)
    w[1] = INV ? cmk<V>(h * (w[1].x - w[1].y), h * (w[1].x + w[1].y))
               : cmk<V>(h * (w[1].x + w[1].y), h * (w[1].y - w[1].x));
    w[2] = rot90<INV>(w[2]);
    w[3] = INV ? cmk<V>(-h * (w[3].x + w[3].y), h * (w[3].x - w[3].y))
               : cmk<V>(h * (w[3].y - w[3].x), -h * (w[3].x + w[3].y));
    dft_small<4, INV>(u);
    dft_small<4, INV>(w);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      v[2 * r] = u[r];
      v[2 * r + 1] = w[r];
    }
  }
}

// One Stockham pass of radix R over a length-2^logm transform in shared memory
// (positions spos): butterfly j (j < M/R) takes elements j + r M/R, multiplies
// element r by W^(k r) with W = exp(-+ 2 pi i / (Ns R)), k = j mod Ns, does the
// length-R DFT and writes element r to (j - k) R + k + r Ns.  Each thread
// handles butterflies threadIdx.x + q blockDim.x, q < Q (blockDim.x * Q * R
// >= M).  tw[j] = exp(-2 pi i j / 2^logtw), j < 2^(logtw-1).
// NZ < R: elements j + r M/R with r >= NZ are zero and not read; NO < R:
// only outputs r < NO are written (radix 16, see dft_small).
template <int R, int Q, bool INV, int NZ = R, int NO = R, typename V>
__device__ __forceinline__ void stockham_pass(V* buf, int logm, int Ns, const V* __restrict__ tw, int logtw,
                                              const V* __restrict__ pre = nullptr) {
  const int nb = (1 << logm) / R;
  // with nb a multiple of 16 the inputs j + r nb sit at spos(j) + r istr; the
  // outputs base + r Ns at spos(base) + r ostr when Ns >= 16 or (radix 16,
  // Ns = 1) base = 16 j
  const bool lin_in = (nb & 15) == 0;
  const int istr = nb + (nb >> 4);
  const bool lin_out = Ns >= 16 || (Ns == 1 && R == 16);
  const int ostr = Ns >= 16 ? Ns + (Ns >> 4) : 1;
  V v[Q][R], wq[Q];
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int j = threadIdx.x + q * blockDim.x;
    if (j < nb) {
      // the butterfly's twiddle W^k, k = j mod Ns (k / (Ns R) < 1/2: inside
      // the stored half of the table), fetched before the barrier
      if (Ns > 1) wq[q] = tw[(j & (Ns - 1)) << (logtw - __ffs(Ns * R) + 1)];
#pragma unroll
      for (int r = NZ; r < R; ++r) v[q][r] = cmk<V>(0, 0);
      if (lin_in) {
        const V* src = buf + spos(j);
#pragma unroll
        for (int r = 0; r < NZ; ++r) v[q][r] = src[r * istr];
      } else {
#pragma unroll
        for (int r = 0; r < NZ; ++r) v[q][r] = buf[spos(j + r * nb)];
      }
      if (pre) {
#pragma unroll
        for (int r = 0; r < NZ; ++r) v[q][r] = cmul(v[q][r], pre[j + r * nb]);  // pointwise product fused into the read
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int j = threadIdx.x + q * blockDim.x;
    if (j < nb) {
      const int k = j & (Ns - 1);
      if (Ns > 1) {
        V w = wq[q];
        if (INV) w.y = -w.y;
        if constexpr (R == 16) {  // w^r from w, w^2, w^4, w^8: at most four products deep
          const V w2 = cmul(w, w), w4 = cmul(w2, w2), w8 = cmul(w4, w4);
          const V w3 = cmul(w2, w), w5 = cmul(w4, w), w6 = cmul(w4, w2), w7 = cmul(w4, w3);
          const V p[8] = {cmk<V>(1, 0), w, w2, w3, w4, w5, w6, w7};
#pragma unroll
          for (int r = 1; r < 8; ++r) {
            v[q][r] = cmul(v[q][r], p[r]);
            v[q][r + 8] = cmul(v[q][r + 8], cmul(w8, p[r]));
          }
          v[q][8] = cmul(v[q][8], w8);
        } else {
          V wr = w;
#pragma unroll
          for (int r = 1; r < R; ++r) {
            v[q][r] = cmul(v[q][r], wr);
            if (r + 1 < R) wr = cmul(wr, w);
          }
        }
      }
      dft_small<R, INV, NZ, NO>(v[q]);
      const int base = (j - k) * R + k;
      if (lin_out) {
        V* dst = buf + spos(base);
#pragma unroll
        for (int r = 0; r < NO; ++r) dst[r * ostr] = v[q][r];
      } else {
#pragma unroll
        for (int r = 0; r < NO; ++r) buf[spos(base + r * Ns)] = v[q][r];
      }
    }
  }
  __syncthreads();
}

// Length-2^logm FFT of buf (positions spos), natural order in and out; needs
// blockDim.x * 16 >= 2^logm.  Caller has synchronised after filling buf.
// The radix-2, -4 or -8 pass comes last: there Ns R = 2^logm, so its writes
// are contiguous.
// `pre`, if given, multiplies the input pointwise as the first pass reads it.
// `first` passes are done already (the caller's own first pass).
// `half_in`: the upper half of the input is zero (the first pass, radix 16,
// neither reads nor transforms it); `half_out`: only the lower half of the
// output is wanted (a last pass of radix 16 writes no other).
template <bool INV, typename V>
__device__ void fft_pow2(V* buf, int logm, const V* __restrict__ tw, int logtw, const V* __restrict__ pre = nullptr,
                         int first = 0, bool half_in = false, bool half_out = false) {
  int Ns = 1 << (4 * first), rest = logm - 4 * first;
  if (half_in && Ns == 1 && rest >= 4) {
    stockham_pass<16, 1, INV, 8, 16>(buf, logm, Ns, tw, logtw, pre);
    Ns <<= 4;
    rest -= 4;
  }
  const bool cut = half_out && (logm & 3) == 0 && rest >= 8;
  for (; rest >= (cut ? 8 : 4); rest -= 4) {
    stockham_pass<16, 1, INV>(buf, logm, Ns, tw, logtw, Ns == 1 ? pre : nullptr);
    Ns <<= 4;
  }
  if (cut) {
    stockham_pass<16, 1, INV, 16, 8>(buf, logm, Ns, tw, logtw, static_cast<const V*>(nullptr));
    Ns <<= 4;
  }
  switch (logm & 3) {
    case 1: stockham_pass<2, 8, INV>(buf, logm, Ns, tw, logtw, Ns == 1 ? pre : nullptr); break;
    case 2: stockham_pass<4, 4, INV>(buf, logm, Ns, tw, logtw, Ns == 1 ? pre : nullptr); break;
    case 3: stockham_pass<8, 2, INV>(buf, logm, Ns, tw, logtw, Ns == 1 ? pre : nullptr); break;
  }
}

// DFT of length H of buf[0..H) (positions spos) in place, natural order: the
// power-of-two FFT when H = 2^logm; otherwise Bluestein's convolution with the
// kernel spectrum Bk (length M = 2^logm >= 2H, natural order, scaled 1/M),
// where the caller has already multiplied buf[n] by the chirp C[n] =
// exp(-pi i n^2 / H) and zero-filled [H, M/2), and multiplies output k < H by
// C[k] as it reads it.  The convolution's input is zero in [M/2, M) and only
// its outputs below H <= M/2 are used, so the first pass of the forward
// transform reads half its inputs and the last pass of the inverse (when it
// is of radix 16) writes half its outputs; [M/2, M) is left undefined.
// Caller has synchronised after filling buf.
template <typename V>
__device__ void ring_dft(V* buf, int logm, bool bluestein, const V* __restrict__ Bk, const V* __restrict__ tw,
                         int logtw) {
  fft_pow2<false>(buf, logm, tw, logtw, static_cast<const V*>(nullptr), 0, bluestein);
  if (bluestein) fft_pow2<true>(buf, logm, tw, logtw, Bk, 0, false, true);
}

// Offset of the chirp table of the cap ring of length N = 4i: i (i - 1).
__device__ __forceinline__ long long chirp_offset(int N) {
  const long long i = N >> 2;
  return i * (i - 1);
}

// Ring of launch slot q: belt launches take y = nside - 1 + q; cap launches
// take the cap rings i = ilo .. ilo + n - 1 (4i pixels) of the north cap
// (y = i - 1), then of the south cap (y = 4 nside - 1 - i).
__device__ __forceinline__ int slot_ring(int q, int caps, int ilo, int n, int nside) {
  if (!caps) return nside - 1 + q;
  return q < n ? ilo + q - 1 : 4 * nside - 1 - (ilo + q - n);
}

// ---------------------------------------------------------------------------
// analysis: real ring -> half spectrum X_y[k], k = 0..N/2 (Eq. 13)
// ---------------------------------------------------------------------------
// Resident CTAs per SM the ring kernels are compiled for: two of 512
// threads (64 registers a thread) in FP32, 512 threads in FP64; the synthesis
// kernel's build for launches of at most 256 threads takes five (48
// registers: c2r 0.86 -> 0.80 ms at Nside 1024, 8 channels; the analysis
// kernel measured no faster there).
template <typename T, int MAXT> constexpr int ring_min_blocks() {
  return sizeof(T) == 8 ? 512 / MAXT : (MAXT <= 256 ? 5 : 1024 / MAXT);
}

template <typename T>
__global__ void __launch_bounds__(512, (ring_min_blocks<T, 512>()))
k_ring_r2c(const T* __restrict__ map, C2<T>* __restrict__ spec, const RingInfo* __restrict__ rings,
           const C2<T>* __restrict__ etab, const C2<T>* __restrict__ btab, const C2<T>* __restrict__ chirp,
           const C2<T>* __restrict__ tw, int logtw, long long npix, long long nspec, int caps, int ilo, int ncap,
           int nside, unsigned* __restrict__ bmax) {
  using V = C2<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* buf = reinterpret_cast<V*>(smem_raw);
  const int y = slot_ring(blockIdx.y, caps, ilo, ncap, nside), b = blockIdx.x;
  const RingInfo R = rings[y];
  const int H = R.nphi >> 1, logm = R.logm;
  const bool blue = R.btab >= 0;
  const V* E = etab + R.etab;
  const V* C = blue ? chirp + chirp_offset(R.nphi) : nullptr;
  // (x[2n], x[2n+1]) as one complex sample z[n]; Bluestein: times the chirp,
  // zero-padded to 2^(logm-1) (the pruned first pass reads no further)
  const V* x2 = reinterpret_cast<const V*>(map + (long long)b * npix + R.start);
  const int M = blue ? 1 << logm : H;
  if (!blue && logm >= 4) {
    // power-of-two rings: the first radix-16 pass (Ns = 1, no twiddles)
    // reads the ring straight from HBM -- butterfly j takes elements
    // j + r H/16, contiguous across the block's threads -- and writes
    // elements 16 j + r: no separate load loop, one shared-memory round trip
    // and one barrier fewer (r2c 0.67 -> 0.58 ms at Nside 1024, 8 channels;
    // the same for the Bluestein rings, or the last pass of c2r written
    // straight to the map, measured slower)
    const int nb = H >> 4;
    for (int j = threadIdx.x; j < nb; j += blockDim.x) {
      V v[16];
#pragma unroll
      for (int r = 0; r < 16; ++r) v[r] = x2[j + r * nb];
      dft_small<16, false>(v);
      const int b0 = spos(16 * j);
#pragma unroll
      for (int r = 0; r < 16; ++r) buf[b0 + r] = v[r];
    }
    __syncthreads();
    fft_pow2<false>(buf, logm, tw, logtw, static_cast<const V*>(nullptr), 1);
  } else {
#pragma unroll 4
    for (int n = threadIdx.x; n < H; n += blockDim.x) buf[spos(n)] = blue ? cmul(x2[n], C[n]) : x2[n];
    for (int n = H + threadIdx.x; n < (blue ? M >> 1 : M); n += blockDim.x) buf[spos(n)] = cmk<V>(0, 0);
    __syncthreads();
    ring_dft(buf, logm, blue, blue ? btab + R.btab : nullptr, tw, logtw);
  }
  // X[k] = (Z[k] + conj Z[H-k]) / 2 + exp(-2 pi i k / N) (Z[k] - conj Z[H-k]) / (2 i),
  // indices of Z mod H.  One thread forms X[k] and X[H-k], k <= H/2, from the
  // same two values: with e, d the two halves and P = E[2k] d / i, X[k] = e + P
  // and, as E[2(H-k)] = E[N-2k] = -conj E[2k], X[H-k] = (e.x - P.x, P.y - e.y).
  V* out = spec + (long long)b * nspec + R.specoff;
  T amax = 0;  // largest |component| written by this thread
  for (int k = threadIdx.x; k <= (H >> 1); k += blockDim.x) {
    const int kc = (k == 0) ? 0 : H - k;
    V zk = buf[spos(k)], zc = buf[spos(kc)];
    if (blue) {
      zk = cmul(zk, C[k]);
      zc = cmul(zc, C[kc]);
    }
    zc = cconj(zc);
    const V e = cscale(cadd(zk, zc), (T)0.5);
    const V d = cscale(csub(zk, zc), (T)0.5);
    const V P = cmul(E[2 * k], cmk<V>(d.y, -d.x));
    const V X = cadd(e, P), Xc = cmk<V>(e.x - P.x, P.y - e.y);
    out[k] = X;
    if (H - k != k) out[H - k] = Xc;
    amax = fmax(amax, fmax(fmax(fabs(X.x), fabs(X.y)), fmax(fabs(Xc.x), fabs(Xc.y))));
  }
  // the channel's largest spectrum component, for the 16-bit operand scale
  // of the tensor-core analysis (float plans only; blockDim is a multiple of 32)
  if constexpr (sizeof(T) == 4) {
    if (bmax) {
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, off));
      if ((threadIdx.x & 31) == 0) atomicMax(bmax + b, __float_as_uint(amax));
    }
  }
}

// ---------------------------------------------------------------------------
// synthesis: F_m(y), m = 0..mmax -> ring values (Eq. 24)
// ---------------------------------------------------------------------------
// The ring's values are p_x = sum_{k<N} D[k] exp(2 pi i k x / N) with
// D[k] = sum_{m = k mod N} F_m e^{i m phi0} + sum_{m = -k mod N, m >= 1}
// conj(F_m e^{i m phi0}) (the aliasing fold; m = 0 contributes Re F_0).
template <typename T, int MAXT>
__global__ void __launch_bounds__(MAXT, (ring_min_blocks<T, MAXT>()))
k_ring_c2r(const C2<T>* __restrict__ F, T* __restrict__ map, const RingInfo* __restrict__ rings,
           const C2<T>* __restrict__ etab, const C2<T>* __restrict__ btab, const C2<T>* __restrict__ chirp,
           const C2<T>* __restrict__ tw, int logtw, long long npix, int nring, int mmax,
           int scale_by_weight, int caps, int ilo, int ncap, int nside) {
  using V = C2<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* buf = reinterpret_cast<V*>(smem_raw);
  const int y = slot_ring(blockIdx.y, caps, ilo, ncap, nside), b = blockIdx.x;
  const RingInfo R = rings[y];
  const int N = R.nphi, H = N >> 1, logm = R.logm, sig = R.sigma;
  const unsigned twoN = 2u * (unsigned)N;  // sigma m < 2^15: 32-bit arithmetic is exact
  const bool blue = R.btab >= 0;
  const V* E = etab + R.etab;
  const V* C = blue ? chirp + chirp_offset(N) : nullptr;
  const V* Fy = F + ((long long)b * nring + y) * (mmax + 1);

  // F_m exp(+i pi sigma m / N) = F_m conj E[ip], ip = sigma m mod 2N.  The
  // aliases of bin k are m = k + t N and m = (t+1) N - k, t >= 0; their phase
  // indices differ from the first one's by t sigma N mod 2N = t step, step =
  // sigma N mod 2N (0 or N), and E[i + N] = -E[i].  So each kind of alias is
  // summed as F (signs alternating in t where step = N), and the sum takes
  // the first alias's phase once: D[k] = phA SA + conj(phB SB).
  auto wrap = [&](unsigned i) { return i >= twoN ? i - twoN : i; };  // i < 4N
  const unsigned step = ((unsigned)sig * (unsigned)N) % twoN;
  const bool alt = step != 0;
  auto fval = [&](int m) {  // F_m, with Im F_0 dropped (real maps)
    V f = Fy[m];
    if (m == 0) f.y = 0;
    return f;
  };
  const int per_bin = (mmax + N) / N;
  if (per_bin > 8) {  // few bins, many aliases: one warp per bin
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    // lane l takes the aliases t = l, l + 32, ...: all of one sign
    const T sgn = (alt && (lane & 1)) ? (T)-1 : (T)1;
    for (int k = warp; k <= H; k += nw) {
      V sa = cmk<V>(0, 0), sb = cmk<V>(0, 0);
      for (int m = k + lane * N; m <= mmax; m += 32 * N) sa = cadd(sa, fval(m));
      for (int m = (lane + 1) * N - k; m <= mmax; m += 32 * N) sb = cadd(sb, Fy[m]);
      sa = cscale(sa, sgn);
      sb = cscale(sb, sgn);
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        sa.x += __shfl_xor_sync(0xffffffffu, sa.x, off);
        sa.y += __shfl_xor_sync(0xffffffffu, sa.y, off);
        sb.x += __shfl_xor_sync(0xffffffffu, sb.x, off);
        sb.y += __shfl_xor_sync(0xffffffffu, sb.y, off);
      }
      if (lane == 0) {
        const unsigned ip = ((unsigned)sig * (unsigned)k) % twoN;
        buf[spos(k)] = cadd(cmul(sa, cconj(E[ip])), cconj(cmul(sb, cconj(E[wrap(step + (twoN - ip))]))));
      }
    }
  } else if (mmax < N) {
    // at most one alias of each kind per bin (m = k and m = N - k): loads of
    // several bins in flight at once
#pragma unroll 4
    for (int k = threadIdx.x; k <= H; k += blockDim.x) {
      unsigned ip = (unsigned)sig * (unsigned)k;
      if (ip >= twoN) ip %= twoN;
      V acc = cmk<V>(0, 0);
      if (k <= mmax) acc = cmul(fval(k), cconj(E[ip]));
      if (N - k <= mmax) acc = cadd(acc, cconj(cmul(Fy[N - k], cconj(E[wrap(step + (twoN - ip))]))));
      buf[spos(k)] = acc;
    }
  } else {
    for (int k = threadIdx.x; k <= H; k += blockDim.x) {
      unsigned ip = (unsigned)sig * (unsigned)k;
      if (ip >= twoN) ip %= twoN;
      // even and odd t apart, then combined with the sign of odd t
      V a0 = cmk<V>(0, 0), a1 = a0, b0 = a0, b1 = a0;
      for (int m = k; m <= mmax; m += 2 * N) {
        a0 = cadd(a0, fval(m));
        if (m + N <= mmax) a1 = cadd(a1, Fy[m + N]);
      }
      for (int m = N - k; m <= mmax; m += 2 * N) {
        b0 = cadd(b0, Fy[m]);
        if (m + N <= mmax) b1 = cadd(b1, Fy[m + N]);
      }
      const V sa = alt ? csub(a0, a1) : cadd(a0, a1), sb = alt ? csub(b0, b1) : cadd(b0, b1);
      buf[spos(k)] = cadd(cmul(sa, cconj(E[ip])), cconj(cmul(sb, cconj(E[wrap(step + (twoN - ip))]))));
    }
  }
  __syncthreads();
  // Z[k] = (D[k] + conj D[H-k]) + i exp(2 pi i k / N) (D[k] - conj D[H-k]), k < H;
  // the ring is then z = IDFT_H(Z) with p[2n] = Re z[n], p[2n+1] = Im z[n].
  // Computed as conj(DFT_H(conj Z)), so conj Z (Bluestein: times the chirp,
  // zero-padded to 2^(logm-1)) is stored.
  if (!blue && logm >= 4 && (H >> 4) <= (int)blockDim.x) {
    // power-of-two rings: conj Z is formed as the first radix-16 pass
    // (Ns = 1) reads its inputs j + r H/16 -- no separate pass over the
    // buffer -- and that pass writes elements 16 j + r
    const int nb = H >> 4, j = threadIdx.x;
    V v[16];
    auto conj_z = [&](V dk, V dc, V e) {
      const V s1 = cadd(dk, cconj(dc)), d1 = csub(dk, cconj(dc));
      const V t1 = cmul(cconj(e), d1);
      return cmk<V>(s1.x - t1.y, -(s1.y + t1.x));
    };
    if (j < nb && (nb & 15) == 0) {
      // k = j + r nb and H - k sit at spos(j) + r istr and spos(H - j) - r istr
      const int istr = nb + (nb >> 4);
      const V *pa = buf + spos(j), *pb = buf + spos(H - j), *ek = E + 2 * j;
#pragma unroll
      for (int r = 0; r < 16; ++r) v[r] = conj_z(pa[r * istr], pb[-r * istr], ek[2 * r * nb]);
    } else if (j < nb) {
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        const int k = j + r * nb;
        v[r] = conj_z(buf[spos(k)], buf[spos(H - k)], E[2 * k]);
      }
    }
    __syncthreads();
    if (j < nb) {
      dft_small<16, false>(v);
      const int b0 = spos(16 * j);
#pragma unroll
      for (int r = 0; r < 16; ++r) buf[b0 + r] = v[r];
    }
    __syncthreads();
    fft_pow2<false>(buf, logm, tw, logtw, static_cast<const V*>(nullptr), 1);
  } else
  {
  for (int k = threadIdx.x; k <= H / 2; k += blockDim.x) {
    const int kc = H - k;
    const V dk = buf[spos(k)], dc = buf[spos(kc)];
    const V s1 = cadd(dk, cconj(dc)), d1 = csub(dk, cconj(dc));
    const V t1 = cmul(cconj(E[2 * k]), d1);
    const V zk = cmk<V>(s1.x - t1.y, s1.y + t1.x);
    if (k > 0 && kc != k) {
      const V s2 = cadd(dc, cconj(dk)), d2 = csub(dc, cconj(dk));
      const V t2 = cmul(cconj(E[2 * kc]), d2);
      const V zc = cmk<V>(s2.x - t2.y, -(s2.y + t2.x));
      buf[spos(kc)] = blue ? cmul(zc, C[kc]) : zc;
    }
    buf[spos(k)] = blue ? cmul(cconj(zk), C[k]) : cconj(zk);
  }
  // zero padding; position H (read above as D[H] for k = 0) is cleared by
  // thread 0 after its own read
  if (blue)
    for (int n = H + threadIdx.x; n < (1 << (logm - 1)); n += blockDim.x) buf[spos(n)] = cmk<V>(0, 0);
  __syncthreads();
  ring_dft(buf, logm, blue, blue ? btab + R.btab : nullptr, tw, logtw);
  }
  const T sc = scale_by_weight ? (T)R.w : (T)1;
  V* out = reinterpret_cast<V*>(map + (long long)b * npix + R.start);
#pragma unroll 4
  for (int n = threadIdx.x; n < H; n += blockDim.x) {
    const V r = blue ? cmul(buf[spos(n)], C[n]) : buf[spos(n)];
    out[n] = cmk<V>(r.x * sc, -r.y * sc);
  }
}

// ---------------------------------------------------------------------------
// plan-time tables
// ---------------------------------------------------------------------------
// E_N[r] = exp(-i pi r / N), r in [0, 2N), for every distinct ring length:
// segment i = 1..nside-1 is the cap ring length 4i (offset 4 i (i - 1)),
// segment nside the belt length 4 nside (offset 4 nside (nside - 1)).
template <typename T>
__global__ void k_build_etab(int nside, C2<T>* etab) {
  const int seg = blockIdx.y + 1;
  const long long N = (seg < nside) ? 4LL * seg : 4LL * nside;
  const long long off = (seg < nside) ? 4LL * seg * (seg - 1) : 4LL * nside * (nside - 1);
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < 2 * N;
       r += (long long)gridDim.x * blockDim.x) {
    double sn, cs;
    sincospi((double)r / (double)N, &sn, &cs);
    etab[off + r] = cmk<C2<T>>((T)cs, (T)(-sn));
  }
}

// Chirp of the cap ring i (H = 2i, N = 4i): C[n] = E_N[2 n^2 mod 2N] =
// exp(-pi i n^2 / H), n < H, at offset i (i - 1) -- the same values the
// E_N table holds, contiguous.
template <typename T>
__global__ void k_build_chirp(int nside, C2<T>* chirp) {
  const int i = blockIdx.y + 1;
  const long long N = 4LL * i, H = 2LL * i;
  for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < H; n += (long long)gridDim.x * blockDim.x) {
    const long long r = (2 * n * n) % (2 * N);
    double sn, cs;
    sincospi((double)r / (double)N, &sn, &cs);
    chirp[(long long)i * (i - 1) + n] = cmk<C2<T>>((T)cs, (T)(-sn));
  }
}

template <typename T>
__global__ void k_build_twiddles(int logtw, C2<T>* tw) {
  const int half = 1 << (logtw - 1);
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < half; j += gridDim.x * blockDim.x) {
    double sn, cs;
    sincospi(-2.0 * (double)j / (double)(1 << logtw), &sn, &cs);
    tw[j] = cmk<C2<T>>((T)cs, (T)sn);
  }
}

// Bluestein kernel spectrum of the cap ring i (H = 2i not a power of two):
// b[j] = exp(+pi i j^2 / H) for |j| < H (indices mod M), zero elsewhere;
// stored as FFT_M(b) / M in natural order.
template <typename T>
__global__ void k_build_bluestein(const RingInfo* __restrict__ rings, const double2* __restrict__ tw64,
                                  int logtw, C2<T>* btab) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* buf = reinterpret_cast<double2*>(smem_raw);
  const RingInfo R = rings[blockIdx.x];  // north cap ring i = blockIdx.x + 1
  if (R.btab < 0) return;                // uniform over the block
  const int H = R.nphi >> 1, M = 1 << R.logm;
  const long long twoN = 4LL * H;
  for (int j = threadIdx.x; j < M; j += blockDim.x) {
    double2 v = cmk<double2>(0.0, 0.0);
    const int jj = (j < H) ? j : ((M - j) < H ? M - j : -1);
    if (jj >= 0) {
      double sn, cs;
      const long long r = (2LL * jj * jj) % twoN;  // pi j^2 / H = pi r / N
      sincospi((double)r / (double)(2 * H), &sn, &cs);
      v = cmk<double2>(cs, sn);
    }
    buf[j] = v;
  }
  __syncthreads();
  fft_dif(buf, R.logm, tw64, logtw, false);
  const double inv = 1.0 / (double)M;
  for (int k = threadIdx.x; k < M; k += blockDim.x) {
    const double2 v = buf[brev(k, R.logm)];  // DIF leaves frequency k at position brev(k)
    btab[R.btab + k] = cmk<C2<T>>((T)(v.x * inv), (T)(v.y * inv));
  }
}

template <typename T>
cudaError_t build_fft_tables(hpx_plan_s* p, cudaStream_t s) {
  using V = C2<T>;
  const int ns = p->nside;
  k_build_etab<T><<<dim3(32, ns), 256, 0, s>>>(ns, (V*)p->d_etab);
  if (ns > 1) k_build_chirp<T><<<dim3(8, ns - 1), 256, 0, s>>>(ns, (V*)p->d_chirp);
  k_build_twiddles<T><<<32, 256, 0, s>>>(p->logtw, (V*)p->d_tw);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (p->nbtab > 0) {
    double2* tw64 = nullptr;
    e = cudaMallocAsync(&tw64, sizeof(double2) << (p->logtw - 1), s);
    if (e != cudaSuccess) return e;
    k_build_twiddles<double><<<32, 256, 0, s>>>(p->logtw, tw64);
    const size_t smem = sizeof(double2) << p->logm_max;
    e = allow_max_smem(k_build_bluestein<T>);
    if (e != cudaSuccess) return e;
    k_build_bluestein<T><<<ns - 1, 256, smem, s>>>(p->d_ring, tw64, p->logtw, (V*)p->d_btab);
    e = cudaGetLastError();
    cudaFreeAsync(tw64, s);
    if (e != cudaSuccess) return e;
  }
  return e;
}

// Launch shapes.  The belt rings (2 nside + 1 of them, H = 2 nside) are one
// launch.  From Nside 512 the cap rings (H = 2i, i < nside; Bluestein length
// 2^L with 4i - 1 <= 2^L < 8i - 2 unless 2i is a power of two) are three, by size:
// the rings of the longest length 2^Lc (i > 2^(Lc-3)), of half that length
// (i > 2^(Lc-4)), and the rest, each launch with the threads and shared
// memory of its own longest transform, so that no CTA carries idle threads
// for a ring a quarter of the launch's size (r2c 0.465 -> 0.440 ms, c2r
// 0.672 -> 0.663 ms at Nside 1024, 8 channels; 3.53 -> 3.29 and 4.71 ->
// 4.38 ms at 64).  The cap launches run on the caller's stream, the belt
// launch on the plan's second stream beside them (the smaller cap classes
// there too measured no faster).
struct RingLaunch {
  int caps, ilo, n, nslots, logm, threads, side;
};
static int fft_threads(int logm) {  // 16 elements per thread at most, 64..512 threads
  int t = (1 << logm) / 16;
  if (t < 64) t = 64;
  return t;
}
static int cap_logm(int i) {  // log2 of the transform length of cap ring i (as the ring table)
  const long long H = 2LL * i;
  long long M = (H & (H - 1)) == 0 ? H : 1;
  if (M == 1)
    while (M < 4LL * i - 1) M <<= 1;
  int L = 0;
  while ((1LL << L) < M) ++L;
  return L;
}
// Below this Nside the transforms are small enough to be bound by launch
// latency (Nside 32: 131 us for an FP64 analysis + synthesis as two launches
// a stage on one stream, 197 us as four on two), and every cap ring fits 64
// threads anyway: one cap launch, no second stream.
constexpr int kSplitNside = 512;

static int ring_launches(const hpx_plan_s* p, RingLaunch* out) {
  const int ns = p->nside;
  int logh = 0;
  while ((1 << logh) < 2 * ns) ++logh;
  int k = 0;
  const bool split = ns >= kSplitNside;
  out[k++] = {0, 0, 0, 2 * ns + 1, logh, fft_threads(logh), split ? 1 : 0};
  if (ns < 2) return k;
  int lc = 0;
  for (int i = 1; i < ns; ++i) lc = cap_logm(i) > lc ? cap_logm(i) : lc;
  if (!split) {  // one launch for all cap rings, everything on the caller's stream
    out[k++] = {1, 1, ns - 1, 2 * (ns - 1), lc, fft_threads(lc), 0};
    return k;
  }
  // i ranges (lo, hi]: (2^(lc-3), ns-1], (2^(lc-4), 2^(lc-3)], (0, 2^(lc-4)]
  int hi = ns - 1;
  for (int c = 0; c < 3 && hi >= 1; ++c) {
    int lo = c < 2 ? (lc - 3 - c >= 0 ? (1 << (lc - 3 - c)) : 0) : 0;
    if (lo > hi) lo = hi;  // nothing in this class
    if (lo < 0) lo = 0;
    if (hi > lo) {
      int L = 0;
      for (int i = lo + 1; i <= hi; ++i) L = cap_logm(i) > L ? cap_logm(i) : L;
      out[k++] = {1, lo + 1, hi - lo, 2 * (hi - lo), L, fft_threads(L), 0};
    }
    hi = lo;
  }
  return k;
}

int ring_launch_count(const hpx_plan_s* p) {
  RingLaunch ls[4];
  return ring_launches(p, ls);
}

static dim3 grid_of(const RingLaunch& L, int nbatch) {
  return dim3(nbatch, L.nslots);  // a ring's channels adjacent: its tables are read once from HBM
}

// The launches of the second stream run beside those on the caller's
// stream: forked from the caller's stream before the launches and joined
// back after them, so the call stays ordered on the caller's stream (and
// captures into a graph as a fork and a join).  `which` picks the stream and
// events of the analysis (0) or the synthesis (1).
struct Fork {
  cudaStream_t s, side;
  cudaEvent_t join_ev = nullptr;
  Fork(const hpx_plan_s* p, int which, cudaStream_t s_, cudaError_t& e) : s(s_), side(s_) {
    if (!p->fft_streams || p->nside < kSplitNside || e != cudaSuccess) return;
    cudaStream_t st = static_cast<cudaStream_t*>(p->fft_streams)[which];
    cudaEvent_t* ev = static_cast<cudaEvent_t*>(p->fft_events) + 2 * which;
    e = cudaEventRecord(ev[0], s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev[0], 0);
    if (e == cudaSuccess) {
      side = st;
      join_ev = ev[1];
    }
  }
  cudaError_t join(cudaError_t e) {
    if (!join_ev) return e;
    cudaError_t e2 = cudaEventRecord(join_ev, side);
    if (e2 == cudaSuccess) e2 = cudaStreamWaitEvent(s, join_ev, 0);
    return e != cudaSuccess ? e : e2;
  }
};

template <typename T>
cudaError_t launch_r2c(const hpx_plan_s* p, const T* map, cudaStream_t s) {
  using V = C2<T>;
  cudaError_t e = allow_max_smem(k_ring_r2c<T>);
  // tensor-core plans with 16-bit operands record each channel's largest
  // spectrum component here (zeroed first)
  unsigned* bmax = (sizeof(T) == 4 && p->tc_mode > 0) ? p->d_bmax : nullptr;
  if (e == cudaSuccess && bmax) e = cudaMemsetAsync(bmax, 0, sizeof(unsigned) * p->nbatch, s);
  Fork f(p, 0, s, e);
  RingLaunch ls[4];
  const int nl = ring_launches(p, ls);
  for (int i = 0; i < nl; ++i) {
    const RingLaunch& L = ls[i];
    if (e != cudaSuccess || L.nslots <= 0) continue;
    k_ring_r2c<T><<<grid_of(L, p->nbatch), L.threads, padded_len(size_t(1) << L.logm) * sizeof(V),
                    L.side ? f.side : s>>>(
        map, (V*)p->d_spec, p->d_ring, (const V*)p->d_etab, (const V*)p->d_btab, (const V*)p->d_chirp,
        (const V*)p->d_tw, p->logtw, p->npix, p->nspec, L.caps, L.ilo, L.n, p->nside, bmax);
    e = cudaGetLastError();
  }
  return f.join(e);
}

template <typename T>
cudaError_t launch_c2r(const hpx_plan_s* p, T* map, bool scale_by_weight, cudaStream_t s) {
  using V = C2<T>;
  cudaError_t e = allow_max_smem(k_ring_c2r<T, 256>);
  if (e == cudaSuccess) e = allow_max_smem(k_ring_c2r<T, 512>);
  Fork f(p, 1, s, e);
  RingLaunch ls[4];
  const int nl = ring_launches(p, ls);
  for (int i = 0; i < nl; ++i) {
    const RingLaunch& L = ls[i];
    if (e != cudaSuccess || L.nslots <= 0) continue;
    auto kern = L.threads <= 256 ? k_ring_c2r<T, 256> : k_ring_c2r<T, 512>;
    kern<<<grid_of(L, p->nbatch), L.threads, padded_len(size_t(1) << L.logm) * sizeof(V), L.side ? f.side : s>>>(
        (const V*)p->d_F, map, p->d_ring, (const V*)p->d_etab, (const V*)p->d_btab, (const V*)p->d_chirp,
        (const V*)p->d_tw, p->logtw, p->npix, p->nring, p->mmax, scale_by_weight ? 1 : 0, L.caps, L.ilo, L.n,
        p->nside);
    e = cudaGetLastError();
  }
  return f.join(e);
}

template cudaError_t build_fft_tables<float>(hpx_plan_s*, cudaStream_t);
template cudaError_t build_fft_tables<double>(hpx_plan_s*, cudaStream_t);
template cudaError_t launch_r2c<float>(const hpx_plan_s*, const float*, cudaStream_t);
template cudaError_t launch_r2c<double>(const hpx_plan_s*, const double*, cudaStream_t);
template cudaError_t launch_c2r<float>(const hpx_plan_s*, float*, bool, cudaStream_t);
template cudaError_t launch_c2r<double>(const hpx_plan_s*, double*, bool, cudaStream_t);

}  // namespace hpx
