// Ring Fourier stage of the HEALPix SHT (Sec. III-D Eq. 13, Sec. III-E).
//
// Every ring y holds N_y = 4i (polar caps) or 4 nside (equatorial belt)
// equally spaced pixels.  A real ring of length N is transformed through a
// complex transform of half length H = N/2 (even samples as real parts, odd
// samples as imaginary parts).  When H is a power of two that transform is a
// radix-2 FFT in shared memory; otherwise it is Bluestein's chirp-z transform
// (Eq. 17-23): chirp multiply, a power-of-two circular convolution done as
// FFT -> pointwise product with the precomputed kernel spectrum -> inverse
// FFT, and a final chirp multiply.  One CTA handles one (ring, channel); the
// whole transform stays in shared memory, so each stage reads its input from
// HBM once and writes its output once.
//
// Chirp and phase angles pi r / N are reduced exactly in integers before the
// FP64 sincospi that fills the tables.
#include "hpx_internal.cuh"

namespace hpx {

__device__ __forceinline__ int brev(int k, int logm) {
  return (int)(__brev((unsigned)k) >> (32 - logm));
}

// Radix-2 decimation in frequency: natural order in, bit-reversed order out.
// tw[j] = exp(-2 pi i j / 2^logtw); inv conjugates the twiddles.
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

// Radix-2 decimation in time: bit-reversed order in, natural order out.
template <typename V>
__device__ void fft_dit(V* buf, int logm, const V* __restrict__ tw, int logtw, bool inv) {
  const int half_n = 1 << (logm - 1);
  for (int s = 0; s < logm; ++s) {
    const int half = 1 << s;
    for (int t = threadIdx.x; t < half_n; t += blockDim.x) {
      const int pos = t & (half - 1);
      const int i0 = ((t >> s) << (s + 1)) + pos;
      const int i1 = i0 + half;
      V w = tw[pos << (logtw - s - 1)];
      if (inv) w.y = -w.y;
      const V a = buf[i0], b = cmul(buf[i1], w);
      buf[i0] = cadd(a, b);
      buf[i1] = csub(a, b);
    }
    __syncthreads();
  }
}

// DFT of length H of buf[0..H) in place, for H = 2^logm (power-of-two case,
// result left in bit-reversed order) or via Bluestein with the kernel
// spectrum Bk of length 2^logm (result in natural order).  E is the ring's
// table exp(-i pi r / N), N = 2H, so the chirp exp(-pi i n^2 / H) is
// E[2 n^2 mod 2N].  Caller has synchronised after filling buf.
template <typename V>
__device__ void ring_dft(V* buf, int H, int logm, bool bluestein, const V* __restrict__ E,
                         const V* __restrict__ Bk, const V* __restrict__ tw, int logtw) {
  // chirp index 2 n^2 mod 2N: n < H <= 8192, so 32-bit unsigned arithmetic is exact
  const unsigned twoN = 4u * (unsigned)H;
  if (!bluestein) {
    fft_dif(buf, logm, tw, logtw, false);
    return;
  }
  const int M = 1 << logm;
  for (int n = threadIdx.x; n < M; n += blockDim.x) {
    if (n < H) buf[n] = cmul(buf[n], E[(2u * (unsigned)n * (unsigned)n) % twoN]);
    else buf[n] = cmk<V>(0, 0);
  }
  __syncthreads();
  fft_dif(buf, logm, tw, logtw, false);
  for (int j = threadIdx.x; j < M; j += blockDim.x) buf[j] = cmul(buf[j], Bk[j]);
  __syncthreads();
  fft_dit(buf, logm, tw, logtw, true);
  for (int k = threadIdx.x; k < H; k += blockDim.x) buf[k] = cmul(buf[k], E[(2u * (unsigned)k * (unsigned)k) % twoN]);
  __syncthreads();
}

// ---------------------------------------------------------------------------
// analysis: real ring -> half spectrum X_y[k], k = 0..N/2 (Eq. 13)
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256)
k_ring_r2c(const T* __restrict__ map, C2<T>* __restrict__ spec, const RingInfo* __restrict__ rings,
           const C2<T>* __restrict__ etab, const C2<T>* __restrict__ btab,
           const C2<T>* __restrict__ tw, int logtw, long long npix, long long nspec) {
  using V = C2<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* buf = reinterpret_cast<V*>(smem_raw);
  const int y = blockIdx.x, b = blockIdx.y;
  const RingInfo R = rings[y];
  const int H = R.nphi >> 1, logm = R.logm;
  const bool blue = R.btab >= 0;
  const V* E = etab + R.etab;
  // (x[2n], x[2n+1]) as one complex sample z[n]
  const V* x2 = reinterpret_cast<const V*>(map + (long long)b * npix + R.start);
  for (int n = threadIdx.x; n < H; n += blockDim.x) buf[n] = x2[n];
  __syncthreads();
  ring_dft(buf, H, logm, blue, E, blue ? btab + R.btab : nullptr, tw, logtw);
  // X[k] = (Z[k] + conj Z[H-k]) / 2 + exp(-2 pi i k / N) (Z[k] - conj Z[H-k]) / (2 i)
  V* out = spec + (long long)b * nspec + R.specoff;
  for (int k = threadIdx.x; k <= H; k += blockDim.x) {
    const int k1 = (k == H) ? 0 : k;
    const int k2 = (k == 0) ? 0 : H - k;
    const V zk = buf[blue ? k1 : brev(k1, logm)];
    const V zc = cconj(buf[blue ? k2 : brev(k2, logm)]);
    const V e = cscale(cadd(zk, zc), (T)0.5);
    const V d = cscale(csub(zk, zc), (T)0.5);
    const V o = cmk<V>(d.y, -d.x);
    out[k] = cadd(e, cmul(E[2 * k], o));
  }
}

// ---------------------------------------------------------------------------
// synthesis: F_m(y), m = 0..mmax -> ring values (Eq. 24)
// ---------------------------------------------------------------------------
// The ring's values are p_x = sum_{k<N} D[k] exp(2 pi i k x / N) with
// D[k] = sum_{m = k mod N} F_m e^{i m phi0} + sum_{m = -k mod N, m >= 1}
// conj(F_m e^{i m phi0}) (the aliasing fold; m = 0 contributes Re F_0).
template <typename T>
__global__ void __launch_bounds__(256)
k_ring_c2r(const C2<T>* __restrict__ F, T* __restrict__ map, const RingInfo* __restrict__ rings,
           const C2<T>* __restrict__ etab, const C2<T>* __restrict__ btab,
           const C2<T>* __restrict__ tw, int logtw, long long npix, int nring, int mmax,
           int scale_by_weight) {
  using V = C2<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* buf = reinterpret_cast<V*>(smem_raw);
  const int y = blockIdx.x, b = blockIdx.y;
  const RingInfo R = rings[y];
  const int N = R.nphi, H = N >> 1, logm = R.logm, sig = R.sigma;
  const unsigned twoN = 2u * (unsigned)N;  // sigma m < 2^15: 32-bit arithmetic is exact
  const bool blue = R.btab >= 0;
  const V* E = etab + R.etab;
  const V* Fy = F + ((long long)b * nring + y) * (mmax + 1);

  auto term = [&](int m) -> V {  // F_m exp(+i pi sigma m / N)
    V f = Fy[m];
    if (m == 0) f.y = 0;
    return cmul(f, cconj(E[((unsigned)sig * (unsigned)m) % twoN]));
  };
  const int per_bin = (mmax + N) / N;
  if (per_bin > 8) {  // few bins, many aliases: one warp per bin
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int k = warp; k <= H; k += nw) {
      V acc = cmk<V>(0, 0);
      for (long long m = k + (long long)lane * N; m <= mmax; m += 32LL * N) acc = cadd(acc, term((int)m));
      for (long long m = N - k + (long long)lane * N; m <= mmax; m += 32LL * N) acc = cadd(acc, cconj(term((int)m)));
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, off);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, off);
      }
      if (lane == 0) buf[k] = acc;
    }
  } else {
    for (int k = threadIdx.x; k <= H; k += blockDim.x) {
      V acc = cmk<V>(0, 0);
      for (int m = k; m <= mmax; m += N) acc = cadd(acc, term(m));
      for (int m = N - k; m <= mmax; m += N) acc = cadd(acc, cconj(term(m)));
      buf[k] = acc;
    }
  }
  __syncthreads();
  // Z[k] = (D[k] + conj D[H-k]) + i exp(2 pi i k / N) (D[k] - conj D[H-k]), k < H;
  // the ring is then z = IDFT_H(Z) with p[2n] = Re z[n], p[2n+1] = Im z[n].
  for (int k = threadIdx.x; k <= H / 2; k += blockDim.x) {
    const int kc = H - k;
    const V dk = buf[k], dc = buf[kc];
    const V s1 = cadd(dk, cconj(dc)), d1 = csub(dk, cconj(dc));
    const V t1 = cmul(cconj(E[2 * k]), d1);
    const V zk = cmk<V>(s1.x - t1.y, s1.y + t1.x);
    if (k > 0 && kc != k) {
      const V s2 = cadd(dc, cconj(dk)), d2 = csub(dc, cconj(dk));
      const V t2 = cmul(cconj(E[2 * kc]), d2);
      buf[kc] = cmk<V>(s2.x - t2.y, s2.y + t2.x);
    }
    buf[k] = zk;
  }
  __syncthreads();
  // IDFT_H(Z) = conj(DFT_H(conj Z))
  for (int n = threadIdx.x; n < H; n += blockDim.x) buf[n] = cconj(buf[n]);
  __syncthreads();
  ring_dft(buf, H, logm, blue, E, blue ? btab + R.btab : nullptr, tw, logtw);
  const T sc = scale_by_weight ? (T)R.w : (T)1;
  V* out = reinterpret_cast<V*>(map + (long long)b * npix + R.start);
  for (int n = threadIdx.x; n < H; n += blockDim.x) {
    const V r = buf[blue ? n : brev(n, logm)];
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
// stored as FFT_M(b) / M in the DIF output order, so the pointwise product
// happens in bit-reversed order between the DIF and DIT passes.
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
  for (int j = threadIdx.x; j < M; j += blockDim.x)
    btab[R.btab + j] = cmk<C2<T>>((T)(buf[j].x * inv), (T)(buf[j].y * inv));
}

template <typename T>
cudaError_t build_fft_tables(hpx_plan_s* p, cudaStream_t s) {
  using V = C2<T>;
  const int ns = p->nside;
  k_build_etab<T><<<dim3(32, ns), 256, 0, s>>>(ns, (V*)p->d_etab);
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

template <typename T>
cudaError_t launch_r2c(const hpx_plan_s* p, const T* map, cudaStream_t s) {
  using V = C2<T>;
  const size_t smem = ((size_t(1) << p->logm_max) + 1) * sizeof(V);
  cudaError_t e = allow_max_smem(k_ring_r2c<T>);
  if (e != cudaSuccess) return e;
  k_ring_r2c<T><<<dim3(p->nring, p->nbatch), 256, smem, s>>>(
      map, (V*)p->d_spec, p->d_ring, (const V*)p->d_etab, (const V*)p->d_btab, (const V*)p->d_tw,
      p->logtw, p->npix, p->nspec);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_c2r(const hpx_plan_s* p, T* map, bool scale_by_weight, cudaStream_t s) {
  using V = C2<T>;
  const size_t smem = ((size_t(1) << p->logm_max) + 1) * sizeof(V);
  cudaError_t e = allow_max_smem(k_ring_c2r<T>);
  if (e != cudaSuccess) return e;
  k_ring_c2r<T><<<dim3(p->nring, p->nbatch), 256, smem, s>>>(
      (const V*)p->d_F, map, p->d_ring, (const V*)p->d_etab, (const V*)p->d_btab, (const V*)p->d_tw,
      p->logtw, p->npix, p->nring, p->mmax, scale_by_weight ? 1 : 0);
  return cudaGetLastError();
}

template cudaError_t build_fft_tables<float>(hpx_plan_s*, cudaStream_t);
template cudaError_t build_fft_tables<double>(hpx_plan_s*, cudaStream_t);
template cudaError_t launch_r2c<float>(const hpx_plan_s*, const float*, cudaStream_t);
template cudaError_t launch_r2c<double>(const hpx_plan_s*, const double*, cudaStream_t);
template cudaError_t launch_c2r<float>(const hpx_plan_s*, float*, bool, cudaStream_t);
template cudaError_t launch_c2r<double>(const hpx_plan_s*, double*, bool, cudaStream_t);

}  // namespace hpx
