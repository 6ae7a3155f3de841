// Data reordering between the HEALPix pixel layouts through the xyf
// representation (Sec. III-B): every layout converts to and from the triplet
// (x, y, f) -- the face f in 0..11 and the position (x, y) in 0..nside-1 on
// it -- and a reorder is source -> xyf -> target.
//
//   RING:   rings north to south, pixels by increasing longitude (Sec. III-A).
//   NESTED: f nside^2 + the Z-order (Morton) interleave of x (even bits) and
//           y (odd bits) within the face.
//   FLAT:   f nside^2 + y nside + x (row-major face images).
//
// Face geometry (Gorski et al. 2005): face f spans the rings around ring
// jr_f nside with jr_f = 2, 3, 4 for the north, equatorial and south faces,
// and its central meridian sits at longitude jp_f pi / 4 with jp_f = 1, 3,
// 5, 7 (polar faces) or 0, 2, 4, 6 (equatorial).  On a face, x + y grows
// northward and x - y eastward: pixel (x, y) lies on ring
// jr = jr_f nside - x - y - 1 (1-based) at 1-based position
// (jp_f nr + x - y + 1 + s) / 2 around it (wrapped into 1..4 nr), nr being
// the ring's pixel count over four and s the belt rings' half-pixel shift
// ((jr - nside) mod 2; 0 on the caps).
//
// The reorder kernel walks the faces in tiles of (x, y): one CTA per face
// and T x T tile (T = min(32, nside)), so no pixel index has to be inverted.
// Each pixel's source and target index follow from its xyf directly; the
// tile's pixels are taken in the order of the target layout (Morton order
// for NESTED, rows for FLAT, the tile's diagonals x + y = const by
// increasing x for RING, each of which is a run of consecutive ring
// pixels), so that a warp's writes are contiguous, and its reads stay within
// the tile, whose source pixels the cache then holds.  All index arithmetic
// is 32-bit (Npix < 2^31 for nside <= 8192).
#include "hpx_internal.cuh"

namespace hpx {
namespace {

__device__ __constant__ int kJr[12] = {2, 2, 2, 2, 3, 3, 3, 3, 4, 4, 4, 4};
__device__ __constant__ int kJp[12] = {1, 3, 5, 7, 0, 2, 4, 6, 1, 3, 5, 7};

struct Xyf {
  int x, y, f;
};

// bits of v spread to the even positions (v < 2^16)
__device__ __forceinline__ unsigned spread_bits(unsigned v) {
  v = (v | (v << 8)) & 0x00FF00FFu;
  v = (v | (v << 4)) & 0x0F0F0F0Fu;
  v = (v | (v << 2)) & 0x33333333u;
  v = (v | (v << 1)) & 0x55555555u;
  return v;
}
// the even-position bits of v packed together
__device__ __forceinline__ unsigned pack_bits(unsigned v) {
  v &= 0x55555555u;
  v = (v | (v >> 1)) & 0x33333333u;
  v = (v | (v >> 2)) & 0x0F0F0F0Fu;
  v = (v | (v >> 4)) & 0x00FF00FFu;
  v = (v | (v >> 8)) & 0x0000FFFFu;
  return v;
}

// ring layout bookkeeping of 1-based ring jr: pixels per quarter, first pixel, shift
struct RingPos {
  long long nr, start;
  int shift;
};
__device__ __forceinline__ RingPos ring_pos(long long nside, long long jr) {
  const long long npix = 12 * nside * nside, ncap = 2 * nside * (nside - 1);
  if (jr < nside) return {jr, 2 * jr * (jr - 1), 0};
  if (jr > 3 * nside) {
    const long long nr = 4 * nside - jr;
    return {nr, npix - 2 * nr * (nr + 1), 0};
  }
  return {nside, ncap + (jr - nside) * 4 * nside, (int)((jr - nside) & 1)};
}

__device__ __forceinline__ long long xyf_to_ring(long long nside, Xyf q) {
  const long long jr = kJr[q.f] * nside - q.x - q.y - 1;
  const RingPos r = ring_pos(nside, jr);
  long long jp = (kJp[q.f] * r.nr + q.x - q.y + 1 + r.shift) / 2;
  if (jp > 4 * r.nr) jp -= 4 * r.nr;
  if (jp < 1) jp += 4 * r.nr;
  return r.start + jp - 1;
}

// Inverse of xyf_to_ring: the ring and position of p give x + y and, up to a
// multiple of 8 nr, x - y for every face; exactly one face puts (x, y) on it.
__device__ __forceinline__ Xyf ring_to_xyf(long long nside, long long p) {
  const long long npix = 12 * nside * nside, ncap = 2 * nside * (nside - 1);
  long long jr, pos;  // 1-based ring, 0-based position
  if (p < ncap) {
    long long i = (long long)((1.0 + sqrt(1.0 + 2.0 * (double)p)) * 0.5);
    while (2 * i * (i - 1) > p) --i;  // exact integer correction of the root
    while (2 * (i + 1) * i <= p) ++i;
    jr = i;
    pos = p - 2 * i * (i - 1);
  } else if (p < npix - ncap) {
    const long long ip = p - ncap;
    jr = ip / (4 * nside) + nside;
    pos = ip % (4 * nside);
  } else {
    const long long ip = npix - 1 - p;
    long long i = (long long)((1.0 + sqrt(1.0 + 2.0 * (double)ip)) * 0.5);
    while (2 * i * (i - 1) > ip) --i;
    while (2 * (i + 1) * i <= ip) ++i;
    jr = 4 * nside - i;
    pos = 2 * i * (i + 1) - 1 - ip;
  }
  const RingPos r = ring_pos(nside, jr);
  const long long jp = pos + 1, period = 8 * r.nr;
  Xyf out{0, 0, -1};
  for (int f = 0; f < 12; ++f) {
    const long long s = kJr[f] * nside - jr - 1;  // x + y
    if (s < 0 || s > 2 * (nside - 1)) continue;
    long long d = 2 * jp - kJp[f] * r.nr - 1 - r.shift;  // x - y, mod 8 nr
    d %= period;
    if (d > period / 2) d -= period;
    if (d < -period / 2) d += period;
    if (((s + d) & 1) != 0) continue;
    const long long x = (s + d) / 2, y = (s - d) / 2;
    if (x >= 0 && x < nside && y >= 0 && y < nside) {
      out = {(int)x, (int)y, f};
      break;
    }
  }
  return out;
}

__device__ __forceinline__ Xyf to_xyf(int layout, long long nside, long long p) {
  if (layout == HPX_RING) return ring_to_xyf(nside, p);
  const long long n2 = nside * nside, f = p / n2, q = p - f * n2;
  if (layout == HPX_NESTED)
    return {(int)pack_bits((unsigned)q), (int)pack_bits((unsigned)(q >> 1)), (int)f};
  return {(int)(q % nside), (int)(q / nside), (int)f};  // FLAT
}

__device__ __forceinline__ long long from_xyf(int layout, long long nside, Xyf q) {
  const long long n2 = nside * nside;
  if (layout == HPX_RING) return xyf_to_ring(nside, q);
  if (layout == HPX_NESTED)
    return q.f * n2 + (long long)(spread_bits((unsigned)q.x) | (spread_bits((unsigned)q.y) << 1));
  return q.f * n2 + (long long)q.y * nside + q.x;  // FLAT
}

// index of pixel q in `layout`, 32-bit (Npix < 2^31)
__device__ __forceinline__ int index_of(int layout, int nside, Xyf q) {
  const int n2 = nside * nside;
  if (layout == HPX_NESTED) return q.f * n2 + (int)(spread_bits((unsigned)q.x) | (spread_bits((unsigned)q.y) << 1));
  if (layout == HPX_FLAT) return q.f * n2 + q.y * nside + q.x;
  // RING: ring jr (1-based) of the face's pixel, then its position around it
  const int jr = kJr[q.f] * nside - q.x - q.y - 1;
  int nr, start, shift = 0;
  if (jr < nside) {
    nr = jr;
    start = 2 * jr * (jr - 1);
  } else if (jr > 3 * nside) {
    nr = 4 * nside - jr;
    start = 12 * n2 - 2 * nr * (nr + 1);
  } else {
    nr = nside;
    start = 2 * nside * (nside - 1) + (jr - nside) * 4 * nside;
    shift = (jr - nside) & 1;
  }
  int jp = (kJp[q.f] * nr + q.x - q.y + 1 + shift) / 2;
  if (jp > 4 * nr) jp -= 4 * nr;
  if (jp < 1) jp += 4 * nr;
  return start + jp - 1;
}

// (x, y) within a T x T tile of the i-th pixel in the target layout's order
__device__ __forceinline__ void tile_pixel(int to, int i, int T, int logT, int& lx, int& ly) {
  if (to == HPX_NESTED) {
    lx = (int)pack_bits((unsigned)i);
    ly = (int)pack_bits((unsigned)i >> 1);
  } else if (to == HPX_FLAT) {
    lx = i & (T - 1);
    ly = i >> logT;
  } else {
    // diagonals c = x + y = 0 .. 2T-2 (lengths 1 .. T .. 1), x increasing
    // along each; the second half is the first mirrored through the centre
    const int half = T * (T + 1) / 2;
    const bool second = i >= half;
    const int k = second ? T * T - 1 - i : i;
    int c = (int)((sqrtf(8.f * (float)k + 1.f) - 1.f) * 0.5f);
    while (c * (c + 1) / 2 > k) --c;
    while ((c + 1) * (c + 2) / 2 <= k) ++c;
    const int pos = k - c * (c + 1) / 2;  // 0 .. c
    if (!second) {
      lx = pos;
      ly = c - pos;
    } else {
      lx = T - 1 - pos;
      ly = T - 1 - (c - pos);
    }
  }
}

// out[b][index_to(q)] = in[b][index_from(q)] for every pixel q, elements of
// E bytes.  Grid: ((nside / T)^2 tiles in Morton order, 12 faces), 256 threads.
template <typename E>
__global__ void __launch_bounds__(256)
k_reorder(const E* __restrict__ in, E* __restrict__ out, int nside, int nbatch, int from, int to, int logT) {
  const int T = 1 << logT, f = blockIdx.y;
  const int x0 = (int)pack_bits(blockIdx.x) << logT, y0 = (int)pack_bits(blockIdx.x >> 1) << logT;
  const long long npix = 12LL * nside * nside;
  for (int i = threadIdx.x; i < T * T; i += blockDim.x) {
    int lx, ly;
    tile_pixel(to, i, T, logT, lx, ly);
    const Xyf q{x0 + lx, y0 + ly, f};
    const E* src = in + index_of(from, nside, q);
    E* dst = out + index_of(to, nside, q);
    int b = 0;
    for (; b + 4 <= nbatch; b += 4) {  // four loads in flight
      const E v0 = src[0], v1 = src[npix], v2 = src[2 * npix], v3 = src[3 * npix];
      dst[0] = v0;
      dst[npix] = v1;
      dst[2 * npix] = v2;
      dst[3 * npix] = v3;
      src += 4 * npix;
      dst += 4 * npix;
    }
    for (; b < nbatch; ++b) {
      *dst = *src;
      src += npix;
      dst += npix;
    }
  }
}

__global__ void k_layout_index(long long* __restrict__ idx, int nside, int from, int to, int* __restrict__ bad) {
  const long long npix = 12LL * nside * nside;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < npix;
       t += (long long)gridDim.x * blockDim.x) {
    const Xyf q = to_xyf(to, nside, t);
    if (q.f < 0) {
      atomicExch(bad, 1);
      idx[t] = -1;
      continue;
    }
    idx[t] = from_xyf(from, nside, q);
  }
}

hpx_status check_layout_args(int nside, hpx_layout from, hpx_layout to) {
  if (nside < 1 || nside > 8192 || (nside & (nside - 1))) {
    set_error("nside must be a power of two in [1, 8192], got %d", nside);
    return HPX_ERR_INVALID;
  }
  if (from < HPX_RING || from > HPX_FLAT || to < HPX_RING || to > HPX_FLAT) {
    set_error("unknown layout");
    return HPX_ERR_INVALID;
  }
  return HPX_OK;
}

int grid_for(long long npix) {
  const long long g = (npix + 255) / 256;
  return (int)(g < 152 * 16 ? g : 152 * 16);
}

// Device word the kernels raise if an index has no xyf (never for valid
// input); one per process, read by hpx_layout_status.
__device__ int g_layout_bad = 0;

}  // namespace
}  // namespace hpx

using namespace hpx;

extern "C" {

hpx_status hpx_reorder(int nside, int nbatch, size_t elem_bytes, hpx_layout from, hpx_layout to, const void* in,
                       void* out, hpx_stream_t stream) {
  hpx_status st = check_layout_args(nside, from, to);
  if (st != HPX_OK) return st;
  if (nbatch < 1 || !in || !out || in == out) {
    set_error("hpx_reorder: need nbatch >= 1 and distinct non-null buffers");
    return HPX_ERR_INVALID;
  }
  if ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) % elem_bytes) {
    set_error("hpx_reorder: buffers must be aligned to the element size");
    return HPX_ERR_INVALID;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int logT = 0;
  while ((1 << logT) < nside && logT < 5) ++logT;  // T = min(32, nside)
  const int per_side = nside >> logT;
  const dim3 grid(per_side * per_side, 12);
  switch (elem_bytes) {
    case 4:
      k_reorder<float><<<grid, 256, 0, s>>>((const float*)in, (float*)out, nside, nbatch, from, to, logT);
      break;
    case 8:
      k_reorder<double><<<grid, 256, 0, s>>>((const double*)in, (double*)out, nside, nbatch, from, to, logT);
      break;
    case 16:
      k_reorder<double2><<<grid, 256, 0, s>>>((const double2*)in, (double2*)out, nside, nbatch, from, to, logT);
      break;
    default:
      set_error("hpx_reorder: elem_bytes must be 4, 8 or 16, got %zu", elem_bytes);
      return HPX_ERR_INVALID;
  }
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HPX_OK : cuda_fail(e, "hpx_reorder");
}

hpx_status hpx_layout_index(int nside, hpx_layout from, hpx_layout to, int64_t* index, hpx_stream_t stream) {
  hpx_status st = check_layout_args(nside, from, to);
  if (st != HPX_OK) return st;
  if (!index) {
    set_error("hpx_layout_index: null index buffer");
    return HPX_ERR_INVALID;
  }
  int* bad = nullptr;
  cudaError_t e = cudaGetSymbolAddress((void**)&bad, g_layout_bad);
  if (e != cudaSuccess) return cuda_fail(e, "hpx_layout_index");
  const long long npix = 12LL * nside * nside;
  k_layout_index<<<grid_for(npix), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      reinterpret_cast<long long*>(index), nside, from, to, bad);
  e = cudaGetLastError();
  return e == cudaSuccess ? HPX_OK : cuda_fail(e, "hpx_layout_index");
}

hpx_status hpx_layout_status(void) {
  int v = 0;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpyFromSymbol(&v, g_layout_bad, sizeof(int));
  if (e == cudaSuccess && v) {
    const int zero = 0;
    e = cudaMemcpyToSymbol(g_layout_bad, &zero, sizeof(int));
  }
  if (e != cudaSuccess) return cuda_fail(e, "hpx_layout_status");
  if (v) {
    set_error("a pixel index had no xyf representation");
    return HPX_ERR_INVALID;
  }
  return HPX_OK;
}

}  // extern "C"
