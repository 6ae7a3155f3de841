// libhpx C ABI: plans, the device-built ring geometry, and the transform
// entry points declared in hpx.h.
#include <cstdarg>
#include <cstddef>
#include <cmath>
#include <cstring>
#include <vector>

#include "hpx_internal.cuh"

namespace hpx {

static thread_local std::string g_err;

void set_error(const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
}

hpx_status cuda_fail(cudaError_t e, const char* what) {
  set_error("%s: %s", what, cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? HPX_ERR_NOMEM : HPX_ERR_CUDA;
}

static bool is_pow2(long long v) { return v > 0 && (v & (v - 1)) == 0; }
static int ilog2(long long v) {
  int r = 0;
  while ((1LL << r) < v) ++r;
  return r;
}
__device__ __forceinline__ int dlog2(long long v) { return 63 - __clzll(v); }
__device__ __forceinline__ long long dnextpow2(long long v) {
  long long r = 1;
  while (r < v) r <<= 1;
  return r;
}

// Ring y of the HEALPix grid (Sec. III-A; pixel centres as defined by
// Gorski et al. 2005).  With the 1-based ring index i = y + 1:
//   polar cap, i < nside: N = 4i, z = 1 - i^2 / (3 nside^2), phi_0 = pi / N;
//   belt, nside <= i <= 3 nside: N = 4 nside, z = (2 nside - i) 2 / (3 nside),
//     phi_0 = s pi / N with s = (i - nside + 1) mod 2;
//   south cap: mirror of the north cap.
// sin(theta) comes from exact integer forms of (1 - z)(1 + z).  Also records
// each ring's offsets into the half-spectrum workspace and the FFT tables.
__global__ void k_ring_geometry(int nside, RingInfo* rings) {
  const int y = blockIdx.x * blockDim.x + threadIdx.x;
  const long long ns = nside, npix = 12 * ns * ns;
  if (y >= 4 * nside - 1) return;
  const long long i = (long long)y + 1;
  const bool south = i > 2 * ns;
  const long long ii = south ? 4 * ns - i : i;
  RingInfo R;
  R.pad = 0;
  if (ii < ns) {
    const double den = 3.0 * (double)(ns * ns);
    R.nphi = (int)(4 * ii);
    R.sigma = 1;
    R.z = 1.0 - (double)(ii * ii) / den;
    R.sinth = (double)ii * sqrt((double)(6 * ns * ns - ii * ii)) / den;
    R.start = south ? npix - 2 * ii * (ii + 1) : 2 * ii * (ii - 1);
    R.specoff = south ? (ns * ns - 1) + (2 * ns + 1) * (2 * ns + 1) + ns * ns - (ii + 1) * (ii + 1)
                      : ii * ii - 1;
    R.etab = 4 * ii * (ii - 1);
    const long long H = 2 * ii;
    if ((ii & (ii - 1)) == 0) {
      R.logm = dlog2(H);
      R.btab = -1;
    } else {
      R.logm = dlog2(dnextpow2(4 * ii - 1));
      long long off = 0;
      for (long long j = 1; j < ii; ++j)
        if ((j & (j - 1)) != 0) off += dnextpow2(4 * j - 1);
      R.btab = off;
    }
  } else {
    R.nphi = (int)(4 * ns);
    R.sigma = (int)((i - ns + 1) & 1);
    R.z = (double)(2 * (2 * ns - ii)) / (double)(3 * ns);
    R.sinth = sqrt((double)((2 * ii - ns) * (7 * ns - 2 * ii))) / (double)(3 * ns);
    R.start = 2 * ns * (ns - 1) + 4 * ns * (i - ns);
    R.specoff = (ns * ns - 1) + (i - ns) * (2 * ns + 1);
    R.etab = 4 * ns * (ns - 1);
    R.logm = dlog2(2 * ns);
    R.btab = -1;
  }
  if (south) R.z = -R.z;
  R.w = (4.0 * 3.14159265358979323846) / (double)npix;
  rings[y] = R;
}

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
  }
};

// Optional per-stage CUDA events (hpx_plan_set_timing).
constexpr int kStages = 6;
struct TimingRec {
  int stage;
  cudaEvent_t a, b;
  int n;
};
struct TimingState {
  bool on = false;
  std::vector<TimingRec> recs;
};

static void plan_free(hpx_plan_s* p) {
  if (!p) return;
  free_tc_host(p);
  for (int k = 0; k < 2; ++k) {
    if (p->d_aio_map[k]) cudaFree(p->d_aio_map[k]);
    if (p->d_aio_alm[k]) cudaFree(p->d_aio_alm[k]);
  }
  if (p->aio_events) {
    cudaEvent_t* ev = static_cast<cudaEvent_t*>(p->aio_events);
    for (int i = 0; i < 6; ++i)
      if (ev[i]) cudaEventDestroy(ev[i]);
    delete[] ev;
  }
  if (p->aio_streams) {
    cudaStream_t* st = static_cast<cudaStream_t*>(p->aio_streams);
    for (int i = 0; i < 2; ++i)
      if (st[i]) cudaStreamDestroy(st[i]);
    delete[] st;
  }
  if (p->fft_events) {
    cudaEvent_t* ev = static_cast<cudaEvent_t*>(p->fft_events);
    for (int i = 0; i < 4; ++i)
      if (ev[i]) cudaEventDestroy(ev[i]);
    delete[] ev;
  }
  if (p->fft_streams) {
    cudaStream_t* st = static_cast<cudaStream_t*>(p->fft_streams);
    for (int i = 0; i < 2; ++i)
      if (st[i]) cudaStreamDestroy(st[i]);
    delete[] st;
  }
  void* ptrs[] = {p->d_ring, p->d_etab, p->d_btab, p->d_chirp, p->d_tw, p->d_cmm, p->d_coef_c, p->d_coef_cf, p->d_coef_p,
                  p->d_coef_pf, p->d_lc, p->d_mu0, p->d_mu1, p->d_spec, p->d_F, p->d_io_map, p->d_io_alm,
                  p->d_tab, p->d_tab_off, p->d_tab_lstart, p->d_gt, p->d_status, p->d_at, p->d_achunk,
                  p->d_stab, p->d_stab_off, p->d_stab_lstart, p->d_tab_lo, p->d_stab_lo, p->d_bmax,
                  p->d_it_map, p->d_it_alm};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  if (p->timing) {
    TimingState* ts = static_cast<TimingState*>(p->timing);
    for (auto& r : ts->recs) {
      cudaEventDestroy(r.a);
      cudaEventDestroy(r.b);
    }
    delete ts;
  }
  delete p;
}

static bool aligned16(const void* ptr) { return (reinterpret_cast<uintptr_t>(ptr) & 15u) == 0; }

static hpx_status check_call(const hpx_plan_s* p, const void* in, const void* out) {
  if (!p) {
    set_error("null plan");
    return HPX_ERR_INVALID;
  }
  if (!in || !out) {
    set_error("null data pointer");
    return HPX_ERR_INVALID;
  }
  if (!aligned16(in) || !aligned16(out)) {
    set_error("data pointers must be 16-byte aligned");
    return HPX_ERR_INVALID;
  }
  return HPX_OK;
}

size_t real_size(const hpx_plan_s* p) { return p->dtype == HPX_F64 ? sizeof(double) : sizeof(float); }

template <class F>
static cudaError_t staged(hpx_plan_s* p, int stage, cudaStream_t s, F&& f) {
  TimingState* ts = static_cast<TimingState*>(p->timing);
  int n = 0;
  if (!ts || !ts->on) return f(&n);
  TimingRec r{stage, nullptr, nullptr, 0};
  cudaError_t e = cudaEventCreate(&r.a);
  if (e == cudaSuccess) e = cudaEventCreate(&r.b);
  if (e == cudaSuccess) e = cudaEventRecord(r.a, s);
  if (e != cudaSuccess) return e;
  e = f(&r.n);
  cudaError_t e2 = cudaEventRecord(r.b, s);
  ts->recs.push_back(r);
  return e != cudaSuccess ? e : e2;
}

// kernel launches of one ring-transform stage (hpx_fft.cu)
int ring_launch_count(const hpx_plan_s* p);

template <typename T>
static cudaError_t run_analysis(hpx_plan_s* p, const void* map, void* alm, bool weighted, double mfac,
                                cudaStream_t s) {
  cudaError_t e = staged(p, 0, s, [&](int* n) {
    *n = ring_launch_count(p);  // belt and cap rings
    return launch_r2c<T>(p, static_cast<const T*>(map), s);
  });
  if (e != cudaSuccess) return e;
  if (p->tc_nn_a) {
    // tensor cores: the operand pack of every channel group (stage 4), then
    // one tile launch over all groups (stage 1)
    const int cp = tc_channels_per_launch(p, false);
    for (int b0 = 0; b0 < p->nbatch && e == cudaSuccess; b0 += cp) {
      const int nb = p->nbatch - b0 < cp ? p->nbatch - b0 : cp;
      e = staged(p, 4, s, [&](int* n) {
        *n = 1;
        return launch_pack_tc(p, b0, nb, weighted, s);
      });
    }
    if (e == cudaSuccess)
      e = staged(p, 1, s, [&](int* n) {
        *n = 1;
        return launch_tile_tc(p, static_cast<float*>(alm), 0, p->nbatch, mfac, s);
      });
    return e;
  }
  return staged(p, 1, s,
                [&](int* n) { return launch_analysis<T>(p, static_cast<T*>(alm), weighted, mfac, s, n); });
}

template <typename T>
static cudaError_t run_synthesis(hpx_plan_s* p, const void* alm, void* map, bool weighted, double mfac,
                                 cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  if (p->tc_nn_s) {
    // tensor cores: the operand pack of every channel group (stage 5), then
    // one tile launch over all groups (stage 2), whose groups share each
    // lambda block through L2
    const int cp = tc_channels_per_launch(p, true);
    for (int b0 = 0; b0 < p->nbatch && e == cudaSuccess; b0 += cp) {
      const int nb = p->nbatch - b0 < cp ? p->nbatch - b0 : cp;
      e = staged(p, 5, s, [&](int* n) {
        *n = p->tc_mode ? 2 : 1;  // 16-bit operands: channel maxima, then the pack
        return launch_pack_at_tc(p, static_cast<const float*>(alm), b0, nb, mfac, s);
      });
    }
    if (e == cudaSuccess)
      e = staged(p, 2, s, [&](int* n) {
        *n = 1;
        return launch_synthesis_tc(p, 0, p->nbatch, s);
      });
  } else {
    e = staged(p, 2, s, [&](int* n) { return launch_synthesis<T>(p, static_cast<const T*>(alm), mfac, s, n); });
  }
  if (e == cudaSuccess)
    e = staged(p, 3, s, [&](int* n) {
      *n = ring_launch_count(p);
      return launch_c2r<T>(p, static_cast<T*>(map), weighted, s);
    });
  return e;
}

static hpx_status transform(hpx_plan p, const void* in, void* out, hpx_stream_t stream, bool analysis,
                            bool weighted, const char* name, double mfac = 1.0) {
  hpx_status st = check_call(p, in, out);
  if (st != HPX_OK) return st;
  DeviceGuard g(p->device);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e;
  if (analysis)
    e = p->dtype == HPX_F64 ? run_analysis<double>(p, in, out, weighted, mfac, s)
                            : run_analysis<float>(p, in, out, weighted, mfac, s);
  else
    e = p->dtype == HPX_F64 ? run_synthesis<double>(p, in, out, weighted, mfac, s)
                            : run_synthesis<float>(p, in, out, weighted, mfac, s);
  if (e != cudaSuccess) return cuda_fail(e, name);
  return HPX_OK;
}

// Iterative refinement (Sec. II-A Eq. 4): r = f - S a, then a += A r.
template <typename T>
__global__ void k_residual(const T* __restrict__ f, T* __restrict__ r, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    r[i] = f[i] - r[i];
}
template <typename T>
__global__ void k_accumulate(T* __restrict__ a, const T* __restrict__ d, long long n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    a[i] += d[i];
}
template <typename T>
static cudaError_t elementwise(bool residual, const void* x, void* y, long long n, cudaStream_t s) {
  const int grid = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  if (residual) k_residual<T><<<grid, 256, 0, s>>>(static_cast<const T*>(x), static_cast<T*>(y), n);
  else k_accumulate<T><<<grid, 256, 0, s>>>(static_cast<T*>(y), static_cast<const T*>(x), n);
  return cudaGetLastError();
}

}  // namespace hpx

using namespace hpx;

extern "C" {

int64_t hpx_nalm(int lmax, int mmax) {
  if (lmax < 0 || mmax < 0 || mmax > lmax) return 0;
  return (int64_t)(mmax + 1) * (lmax + 1) - (int64_t)mmax * (mmax + 1) / 2;
}

const char* hpx_last_error(void) { return g_err.c_str(); }

static hpx_status create_plan(int nside, int lmax, int mmax, int nbatch, hpx_dtype dtype, unsigned flags,
                              size_t stage_bytes, hpx_plan* out);

hpx_status hpx_plan_create_ex(int nside, int lmax, int mmax, int nbatch, hpx_dtype dtype, unsigned flags,
                              hpx_plan* out) {
  return create_plan(nside, lmax, mmax, nbatch, dtype, flags, 0, out);
}

hpx_status hpx_plan_create_ooc(int nside, int lmax, int mmax, int nbatch, hpx_dtype dtype, size_t stage_bytes,
                               hpx_plan* out) {
  return create_plan(nside, lmax, mmax, nbatch, dtype,
                     HPX_PLAN_LAMBDA_TABLE | HPX_PLAN_TENSOR_CORES | HPX_PLAN_LAMBDA_HOST, stage_bytes, out);
}

hpx_status hpx_plan_create_stream(int nside, int lmax, int mmax, int nbatch, hpx_dtype dtype, unsigned flags,
                                  size_t stage_bytes, hpx_plan* out) {
  if (flags & ~HPX_PLAN_TC_TF32X3) {
    if (out) *out = nullptr;
    set_error("hpx_plan_create_stream: flags 0x%x (only HPX_PLAN_TC_TF32X3 may be added)", flags);
    return HPX_ERR_INVALID;
  }
  return create_plan(nside, lmax, mmax, nbatch, dtype,
                     flags | HPX_PLAN_LAMBDA_TABLE | HPX_PLAN_TENSOR_CORES | HPX_PLAN_LAMBDA_STREAM, stage_bytes, out);
}

static hpx_status create_plan(int nside, int lmax, int mmax, int nbatch, hpx_dtype dtype, unsigned flags,
                              size_t stage_bytes, hpx_plan* out) {
  if (!out) {
    set_error("null output pointer");
    return HPX_ERR_INVALID;
  }
  *out = nullptr;
  if (nside < 1 || nside > 2048 || !is_pow2(nside)) {
    set_error("nside must be a power of two in [1, 2048], got %d", nside);
    return HPX_ERR_INVALID;
  }
  if (lmax < 0 || lmax > 16384 || mmax < 0 || mmax > lmax) {
    set_error("need 0 <= mmax <= lmax <= 16384, got lmax %d mmax %d", lmax, mmax);
    return HPX_ERR_INVALID;
  }
  if (nbatch < 1 || nbatch > 65535) {
    set_error("nbatch must be in [1, 65535], got %d", nbatch);
    return HPX_ERR_INVALID;
  }
  if (dtype < HPX_F64 || dtype > HPX_F32_FP16X3) {
    set_error("unknown dtype %d", (int)dtype);
    return HPX_ERR_INVALID;
  }
  if (flags & ~(HPX_PLAN_LAMBDA_TABLE | HPX_PLAN_TENSOR_CORES | HPX_PLAN_LAMBDA_HOST | HPX_PLAN_TC_TF32X3 |
                HPX_PLAN_LAMBDA_STREAM)) {
    set_error("unknown plan flags 0x%x", flags);
    return HPX_ERR_INVALID;
  }
  const bool mixed = dtype != HPX_F64 && dtype != HPX_F32;
  if ((flags & HPX_PLAN_TC_TF32X3) && (mixed || !(flags & HPX_PLAN_TENSOR_CORES))) {
    set_error("HPX_PLAN_TC_TF32X3 needs an HPX_F32 plan with HPX_PLAN_TENSOR_CORES");
    return HPX_ERR_INVALID;
  }
  if (mixed) {
    flags = HPX_PLAN_LAMBDA_TABLE | HPX_PLAN_TENSOR_CORES |
            (flags & (HPX_PLAN_LAMBDA_HOST | HPX_PLAN_LAMBDA_STREAM));  // their only path
  } else if ((flags & HPX_PLAN_TENSOR_CORES) && (dtype != HPX_F32 || !(flags & HPX_PLAN_LAMBDA_TABLE))) {
    set_error("HPX_PLAN_TENSOR_CORES needs an HPX_F32 plan with HPX_PLAN_LAMBDA_TABLE");
    return HPX_ERR_INVALID;
  }
  if ((flags & HPX_PLAN_LAMBDA_HOST) && !(flags & HPX_PLAN_TENSOR_CORES)) {
    set_error("HPX_PLAN_LAMBDA_HOST needs the tensor-core path (HPX_PLAN_TENSOR_CORES or a 16-bit dtype)");
    return HPX_ERR_INVALID;
  }
  if ((flags & HPX_PLAN_LAMBDA_STREAM) && !(flags & HPX_PLAN_TENSOR_CORES)) {
    set_error("HPX_PLAN_LAMBDA_STREAM needs the tensor-core path (HPX_PLAN_TENSOR_CORES or a 16-bit dtype)");
    return HPX_ERR_INVALID;
  }
  if ((flags & HPX_PLAN_LAMBDA_STREAM) && (flags & HPX_PLAN_LAMBDA_HOST)) {
    set_error("HPX_PLAN_LAMBDA_STREAM and HPX_PLAN_LAMBDA_HOST exclude each other");
    return HPX_ERR_INVALID;
  }
  hpx_plan_s* p = new hpx_plan_s();
  std::memset(p, 0, sizeof(*p));
  cudaGetDevice(&p->device);
  p->nside = nside;
  p->lmax = lmax;
  p->mmax = mmax;
  p->nbatch = nbatch;
  p->dtype = dtype;
  p->flags = flags;
  p->stage_bytes = stage_bytes;
  p->nring = 4 * nside - 1;
  p->w_max = 4.0 * 3.14159265358979323846 / (12.0 * (double)nside * (double)nside);
  p->npair = 2 * nside;
  p->npix = 12LL * nside * nside;
  p->nalm = hpx_nalm(lmax, mmax);
  p->nspec = 6LL * nside * nside + 4LL * nside - 1;
  p->netab = 4LL * nside * (nside - 1) + 8LL * nside;
  p->nbtab = 0;
  p->logm_max = ilog2(2LL * nside);
  for (long long i = 1; i < nside; ++i) {
    if (is_pow2(i)) continue;
    long long M = 1;
    while (M < 4 * i - 1) M <<= 1;
    p->nbtab += M;
    if (ilog2(M) > p->logm_max) p->logm_max = ilog2(M);
  }
  p->logtw = p->logm_max;
  const size_t rs = real_size(p), cs = 2 * rs;
  const long long nchain = (long long)(mmax + 1) * p->npair;

  auto alloc = [&](void** ptr, size_t bytes) -> bool {
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(ptr, bytes);
    if (e != cudaSuccess) {
      cuda_fail(e, "cudaMalloc");
      *ptr = nullptr;
      return false;
    }
    p->bytes += bytes;
    return true;
  };
  bool ok = alloc((void**)&p->d_ring, sizeof(RingInfo) * p->nring) &&
            alloc(&p->d_etab, cs * p->netab) && alloc(&p->d_btab, cs * p->nbtab) &&
            alloc(&p->d_chirp, cs * (size_t)nside * (nside - 1)) &&
            alloc(&p->d_tw, cs * ((size_t)1 << (p->logtw - 1))) &&
            alloc((void**)&p->d_cmm, sizeof(double) * (mmax + 1)) &&
            alloc((void**)&p->d_coef_c, sizeof(double) * p->nalm) &&
            alloc((void**)&p->d_coef_cf, sizeof(float2) * p->nalm) &&
            alloc((void**)&p->d_coef_p, sizeof(double) * p->nalm) &&
            alloc((void**)&p->d_coef_pf, sizeof(float) * p->nalm) &&
            alloc((void**)&p->d_lc, sizeof(int) * nchain) && alloc((void**)&p->d_mu0, sizeof(double) * nchain) &&
            alloc((void**)&p->d_mu1, sizeof(double) * nchain) &&
            alloc(&p->d_spec, cs * (size_t)nbatch * p->nspec) &&
            alloc(&p->d_F, cs * (size_t)nbatch * p->nring * (mmax + 1)) &&
            alloc((void**)&p->d_status, sizeof(int));
  if (!ok) {
    plan_free(p);
    return HPX_ERR_NOMEM;
  }
  cudaStream_t s;
  cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    plan_free(p);
    return cuda_fail(e, "cudaStreamCreate");
  }
  {
    // the ring transforms' second stream (belt rings beside the cap rings)
    // and its fork / join events; kept by the plan once all of them exist
    cudaStream_t* fs = new cudaStream_t[2]();
    cudaEvent_t* fe = new cudaEvent_t[4]();
    p->fft_streams = fs;
    p->fft_events = fe;
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaStreamCreateWithFlags(&fs[i], cudaStreamNonBlocking);
    for (int i = 0; i < 4 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&fe[i], cudaEventDisableTiming);
    if (e != cudaSuccess) {
      cudaStreamDestroy(s);
      plan_free(p);
      return cuda_fail(e, "ring-transform streams");
    }
  }
  e = cudaMemsetAsync(p->d_status, 0, sizeof(int), s);
  if (e == cudaSuccess) {
    k_ring_geometry<<<(p->nring + 127) / 128, 128, 0, s>>>(nside, p->d_ring);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = build_recurrence_tables(p, s);
  // the CUDA-core table, also the 3xTF32 path's row table; the 16-bit
  // tensor-core paths build their own
  if (e == cudaSuccess && (flags & HPX_PLAN_LAMBDA_TABLE) && tc_mode_of(dtype, flags) <= 0 &&
      !(flags & (HPX_PLAN_LAMBDA_HOST | HPX_PLAN_LAMBDA_STREAM)))
    e = dtype == HPX_F64 ? build_lambda_table<double>(p, s) : build_lambda_table<float>(p, s);
  if (e == cudaSuccess && (flags & HPX_PLAN_TENSOR_CORES)) e = build_tc(p, s);
  if (e == cudaSuccess) e = dtype == HPX_F64 ? build_fft_tables<double>(p, s) : build_fft_tables<float>(p, s);
  cudaError_t e2 = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = e2;
  cudaStreamDestroy(s);
  if (e != cudaSuccess) {
    plan_free(p);
    return cuda_fail(e, "plan construction");
  }
  *out = p;
  return HPX_OK;
}

hpx_status hpx_plan_create(int nside, int lmax, int mmax, int nbatch, hpx_dtype dtype, hpx_plan* out) {
  return hpx_plan_create_ex(nside, lmax, mmax, nbatch, dtype, HPX_PLAN_LAMBDA_RECOMPUTE, out);
}

hpx_status hpx_plan_destroy(hpx_plan plan) {
  if (!plan) return HPX_OK;
  DeviceGuard g(plan->device);
  cudaDeviceSynchronize();
  plan_free(plan);
  return HPX_OK;
}

size_t hpx_plan_device_bytes(hpx_plan plan) { return plan ? plan->bytes : 0; }

size_t hpx_plan_estimate_bytes(int nside, int lmax, int mmax, int nbatch, hpx_dtype dtype, unsigned flags) {
  if (nside < 1 || nside > 2048 || !is_pow2(nside) || lmax < 0 || mmax < 0 || mmax > lmax || nbatch < 1)
    return 0;
  const size_t rs = dtype == HPX_F64 ? sizeof(double) : sizeof(float), cs = 2 * rs;
  const size_t nring = 4 * (size_t)nside - 1, npair = 2 * (size_t)nside;
  const size_t nalm = (size_t)hpx_nalm(lmax, mmax), nchain = (size_t)(mmax + 1) * npair;
  const size_t nspec = 6 * (size_t)nside * nside + 4 * (size_t)nside - 1;
  const size_t netab = 4 * (size_t)nside * (nside - 1) + 8 * (size_t)nside;
  size_t nbtab = 0;
  int logm_max = ilog2(2LL * nside);
  for (long long i = 1; i < nside; ++i) {
    if (is_pow2(i)) continue;
    long long M = 1;
    while (M < 4 * i - 1) M <<= 1;
    nbtab += (size_t)M;
    if (ilog2(M) > logm_max) logm_max = ilog2(M);
  }
  size_t b = sizeof(RingInfo) * nring + cs * netab + cs * (nbtab ? nbtab : 1) + cs * ((size_t)1 << (logm_max - 1)) +
             cs * (size_t)nside * (nside - 1) +
             sizeof(double) * (mmax + 1) + (3 * sizeof(double) + sizeof(float)) * nalm +
             (sizeof(int) + 2 * sizeof(double)) * nchain + cs * (size_t)nbatch * nspec +
             cs * (size_t)nbatch * nring * (mmax + 1);
  const size_t ngroup = (npair + 31) / 32;
  const int mode = tc_mode_of(dtype, flags);
  if (flags & (HPX_PLAN_LAMBDA_HOST | HPX_PLAN_LAMBDA_STREAM))  // no resident table; two staging buffers
    return b + sizeof(int) + tc_extra_bytes_estimate(nside, lmax, mmax, nbatch, mode, true);
  if (mode > 0) return b + sizeof(int) + tc_extra_bytes_estimate(nside, lmax, mmax, nbatch, mode, false);
  if (flags & HPX_PLAN_LAMBDA_TABLE)  // upper bound: every (l, m, ring pair) stored
    b += rs * nalm * npair + (sizeof(int) + sizeof(long long)) * (size_t)(mmax + 1) * ngroup;
  if (flags & HPX_PLAN_TENSOR_CORES)  // row-table starts padded to the tile grid; column table; operands
    b += rs * (size_t)(mmax + 1) * ngroup * 32 * (kTcTile - 1) +
         tc_extra_bytes_estimate(nside, lmax, mmax, nbatch, mode, false);
  return b + sizeof(int);
}

size_t hpx_plan_table_bytes(hpx_plan plan) {
  if (!plan || (!plan->d_tab && !plan->h_tab)) return 0;
  const size_t es = plan->dtype == HPX_F64 ? sizeof(double) : plan->tc_mode > 0 ? 2 : sizeof(float);
  const size_t parts = (plan->d_tab_lo || plan->h_tab_lo) ? 2 : 1;
  return (size_t)plan->tab_elems * es * parts;
}

size_t hpx_plan_column_table_bytes(hpx_plan plan) {
  if (!plan || (!plan->d_stab && !plan->h_stab)) return 0;
  const size_t es = plan->tc_mode > 0 ? 2 : sizeof(float);
  const size_t parts = (plan->d_stab_lo || plan->h_stab_lo) ? 2 : 1;
  return (size_t)plan->stab_elems * es * parts;
}

size_t hpx_plan_host_bytes(hpx_plan plan) { return plan ? plan->host_bytes : 0; }

hpx_status hpx_map2alm(hpx_plan plan, const void* map, void* alm, hpx_stream_t stream) {
  return transform(plan, map, alm, stream, true, true, "hpx_map2alm");
}

hpx_status hpx_alm2map_adjoint(hpx_plan plan, const void* map, void* alm, hpx_stream_t stream) {
  return transform(plan, map, alm, stream, true, false, "hpx_alm2map_adjoint");
}

hpx_status hpx_alm2map(hpx_plan plan, const void* alm, void* map, hpx_stream_t stream) {
  return transform(plan, alm, map, stream, false, false, "hpx_alm2map");
}

hpx_status hpx_map2alm_adjoint(hpx_plan plan, const void* alm, void* map, hpx_stream_t stream) {
  return transform(plan, alm, map, stream, false, true, "hpx_map2alm_adjoint");
}

// The first n channels of the plan's batch: a view of the plan with nbatch n
// (the workspace is channel-major, so its first n channel slices serve).
static hpx_status transform_n(hpx_plan plan, int n, const void* in, void* out, hpx_stream_t stream,
                              bool analysis, const char* name) {
  if (!plan) {
    set_error("%s: null plan", name);
    return HPX_ERR_INVALID;
  }
  if (n < 1 || n > plan->nbatch) {
    set_error("%s: n = %d outside [1, %d]", name, n, plan->nbatch);
    return HPX_ERR_INVALID;
  }
  hpx_plan_s view = *plan;
  view.nbatch = n;
  return transform(&view, in, out, stream, analysis, analysis, name);
}

hpx_status hpx_map2alm_n(hpx_plan plan, int n, const void* map, void* alm, hpx_stream_t stream) {
  return transform_n(plan, n, map, alm, stream, true, "hpx_map2alm_n");
}

hpx_status hpx_alm2map_n(hpx_plan plan, int n, const void* alm, void* map, hpx_stream_t stream) {
  return transform_n(plan, n, alm, map, stream, false, "hpx_alm2map_n");
}

hpx_status hpx_alm2map_grad(hpx_plan plan, const void* grad_map, void* grad_alm, hpx_stream_t stream) {
  return transform(plan, grad_map, grad_alm, stream, true, false, "hpx_alm2map_grad", 2.0);
}

hpx_status hpx_map2alm_grad(hpx_plan plan, const void* grad_alm, void* grad_map, hpx_stream_t stream) {
  return transform(plan, grad_alm, grad_map, stream, false, true, "hpx_map2alm_grad", 0.5);
}

// Reads and clears the plan's device-side wait status (after a sync).
static hpx_status read_status(hpx_plan p) {
  int st = 0;
  cudaError_t e = cudaMemcpy(&st, p->d_status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && st != 0) e = cudaMemset(p->d_status, 0, sizeof(int));
  if (e != cudaSuccess) return cuda_fail(e, "reading the device status");
  if (st != 0) {
    set_error("a bounded device-side wait expired; the transform's output is incomplete");
    return HPX_ERR_TIMEOUT;
  }
  return HPX_OK;
}

static hpx_status host_call(hpx_plan p, const void* hin, void* hout, hpx_stream_t stream, bool analysis) {
  if (!p || !hin || !hout) {
    set_error("null argument");
    return HPX_ERR_INVALID;
  }
  DeviceGuard g(p->device);
  const size_t rs = real_size(p);
  const size_t map_bytes = rs * (size_t)p->nbatch * p->npix;
  const size_t alm_bytes = 2 * rs * (size_t)p->nbatch * p->nalm;
  if (!p->d_io_map) {
    cudaError_t e = cudaMalloc(&p->d_io_map, map_bytes);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc (host I/O buffer)");
    p->bytes += map_bytes;
  }
  if (!p->d_io_alm) {
    cudaError_t e = cudaMalloc(&p->d_io_alm, alm_bytes);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc (host I/O buffer)");
    p->bytes += alm_bytes;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  void* din = analysis ? p->d_io_map : p->d_io_alm;
  void* dout = analysis ? p->d_io_alm : p->d_io_map;
  const size_t in_bytes = analysis ? map_bytes : alm_bytes, out_bytes = analysis ? alm_bytes : map_bytes;
  cudaError_t e = cudaMemcpyAsync(din, hin, in_bytes, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_fail(e, "host-to-device copy");
  hpx_status st = analysis ? hpx_map2alm(p, din, dout, stream) : hpx_alm2map(p, din, dout, stream);
  if (st != HPX_OK) return st;
  e = cudaMemcpyAsync(hout, dout, out_bytes, cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return cuda_fail(e, "device-to-host copy");
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "stream synchronise");
  return read_status(p);
}

// Pipelined host-buffer call: the upload of the input goes on the plan's
// host-to-device stream into I/O slot k (once the call that last used slot k
// has downloaded its result), the transform on `stream` after the upload, and
// the download of the result on the device-to-host stream after the
// transform.  Consecutive calls alternate slots, so one call's copies overlap
// the neighbouring calls' kernels in both directions.
static hpx_status host_call_async(hpx_plan p, const void* hin, void* hout, hpx_stream_t stream, bool analysis) {
  if (!p || !hin || !hout) {
    set_error("null argument");
    return HPX_ERR_INVALID;
  }
  DeviceGuard g(p->device);
  const size_t rs = real_size(p);
  const size_t map_bytes = rs * (size_t)p->nbatch * p->npix;
  const size_t alm_bytes = 2 * rs * (size_t)p->nbatch * p->nalm;
  cudaError_t e = cudaSuccess;
  if (!p->aio_streams) {
    // Everything is made into locals first and handed to the plan only once
    // all of it exists; on a failure what was made is released again, so a
    // later call retries the whole set-up.
    cudaStream_t* st = new cudaStream_t[2]();
    cudaEvent_t* ev = new cudaEvent_t[6]();
    void* dm[2] = {nullptr, nullptr};
    void* da[2] = {nullptr, nullptr};
    for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaStreamCreateWithFlags(&st[i], cudaStreamNonBlocking);
    for (int i = 0; i < 6 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
    for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
      e = cudaMalloc(&dm[k], map_bytes);
      if (e == cudaSuccess) e = cudaMalloc(&da[k], alm_bytes);
    }
    if (e != cudaSuccess) {
      for (int k = 0; k < 2; ++k) {
        if (dm[k]) cudaFree(dm[k]);
        if (da[k]) cudaFree(da[k]);
      }
      for (int i = 0; i < 6; ++i)
        if (ev[i]) cudaEventDestroy(ev[i]);
      for (int i = 0; i < 2; ++i)
        if (st[i]) cudaStreamDestroy(st[i]);
      delete[] ev;
      delete[] st;
      return cuda_fail(e, "pipelined I/O set-up");
    }
    for (int k = 0; k < 2; ++k) {
      p->d_aio_map[k] = dm[k];
      p->d_aio_alm[k] = da[k];
    }
    p->bytes += 2 * (map_bytes + alm_bytes);
    p->aio_events = ev;
    p->aio_streams = st;
  }
  cudaStream_t* st = static_cast<cudaStream_t*>(p->aio_streams);
  cudaEvent_t* ev = static_cast<cudaEvent_t*>(p->aio_events);  // uploaded[2], computed[2], free[2]
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int k = p->aio_next;
  p->aio_next ^= 1;
  void* din = analysis ? p->d_aio_map[k] : p->d_aio_alm[k];
  void* dout = analysis ? p->d_aio_alm[k] : p->d_aio_map[k];
  const size_t in_bytes = analysis ? map_bytes : alm_bytes, out_bytes = analysis ? alm_bytes : map_bytes;
  e = cudaStreamWaitEvent(st[0], ev[4 + k], 0);  // slot k's previous result downloaded
  if (e == cudaSuccess) e = cudaMemcpyAsync(din, hin, in_bytes, cudaMemcpyHostToDevice, st[0]);
  if (e == cudaSuccess) e = cudaEventRecord(ev[k], st[0]);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev[k], 0);
  if (e != cudaSuccess) return cuda_fail(e, "pipelined upload");
  hpx_status r = analysis ? hpx_map2alm(p, din, dout, stream) : hpx_alm2map(p, din, dout, stream);
  if (r != HPX_OK) return r;
  e = cudaEventRecord(ev[2 + k], s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(st[1], ev[2 + k], 0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hout, dout, out_bytes, cudaMemcpyDeviceToHost, st[1]);
  if (e == cudaSuccess) e = cudaEventRecord(ev[4 + k], st[1]);
  if (e != cudaSuccess) return cuda_fail(e, "pipelined download");
  return HPX_OK;
}

hpx_status hpx_map2alm_iter(hpx_plan p, const void* map, void* alm, int niter, hpx_stream_t stream) {
  hpx_status st = check_call(p, map, alm);
  if (st != HPX_OK) return st;
  if (niter < 0 || niter > 1000) {
    set_error("hpx_map2alm_iter: niter must be in [0, 1000], got %d", niter);
    return HPX_ERR_INVALID;
  }
  st = hpx_map2alm(p, map, alm, stream);
  if (st != HPX_OK || niter == 0) return st;
  DeviceGuard g(p->device);
  const size_t rs = real_size(p);
  const long long nmap = (long long)p->nbatch * p->npix, nalm2 = 2LL * p->nbatch * p->nalm;
  if (!p->d_it_map) {
    cudaError_t e = cudaMalloc(&p->d_it_map, rs * nmap);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc (refinement buffer)");
    p->bytes += rs * nmap;
  }
  if (!p->d_it_alm) {
    cudaError_t e = cudaMalloc(&p->d_it_alm, rs * nalm2);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc (refinement buffer)");
    p->bytes += rs * nalm2;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const bool f64 = p->dtype == HPX_F64;
  for (int k = 0; k < niter; ++k) {
    st = hpx_alm2map(p, alm, p->d_it_map, stream);  // S a
    if (st != HPX_OK) return st;
    cudaError_t e = f64 ? elementwise<double>(true, map, p->d_it_map, nmap, s)
                        : elementwise<float>(true, map, p->d_it_map, nmap, s);  // r = f - S a
    if (e != cudaSuccess) return cuda_fail(e, "hpx_map2alm_iter");
    st = hpx_map2alm(p, p->d_it_map, p->d_it_alm, stream);  // A r
    if (st != HPX_OK) return st;
    e = f64 ? elementwise<double>(false, p->d_it_alm, alm, nalm2, s)
            : elementwise<float>(false, p->d_it_alm, alm, nalm2, s);  // a += A r
    if (e != cudaSuccess) return cuda_fail(e, "hpx_map2alm_iter");
  }
  return HPX_OK;
}

hpx_status hpx_plan_set_ring_weights(hpx_plan p, const double* w, int n) {
  if (!p || !w) {
    set_error("null argument");
    return HPX_ERR_INVALID;
  }
  if (n != p->nring) {
    set_error("hpx_plan_set_ring_weights: need %d weights (one per ring), got %d", p->nring, n);
    return HPX_ERR_INVALID;
  }
  double wmax = 0.0;
  for (int y = 0; y < n; ++y) {
    if (!(w[y] == w[y]) || w[y] > 1e300 || w[y] < -1e300) {
      set_error("hpx_plan_set_ring_weights: weight %d is not finite", y);
      return HPX_ERR_INVALID;
    }
    wmax = fmax(wmax, fabs(w[y]));
  }
  DeviceGuard g(p->device);
  // the w field of every RingInfo, one strided copy
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess)
    e = cudaMemcpy2D(reinterpret_cast<char*>(p->d_ring) + offsetof(RingInfo, w), sizeof(RingInfo), w, sizeof(double),
                     sizeof(double), (size_t)n, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "hpx_plan_set_ring_weights");
  p->w_max = wmax;
  return HPX_OK;
}

hpx_status hpx_plan_device_status(hpx_plan plan) {
  if (!plan) {
    set_error("null plan");
    return HPX_ERR_INVALID;
  }
  DeviceGuard g(plan->device);
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "device synchronise");
  return read_status(plan);
}

hpx_status hpx_plan_test_withhold_copies(hpx_plan plan, int withhold) {
  if (!plan) {
    set_error("null plan");
    return HPX_ERR_INVALID;
  }
  plan->test_withhold = withhold ? 1 : 0;
  return HPX_OK;
}

hpx_status hpx_map2alm_host_async(hpx_plan plan, const void* host_map, void* host_alm, hpx_stream_t stream) {
  return host_call_async(plan, host_map, host_alm, stream, true);
}

hpx_status hpx_alm2map_host_async(hpx_plan plan, const void* host_alm, void* host_map, hpx_stream_t stream) {
  return host_call_async(plan, host_alm, host_map, stream, false);
}

hpx_status hpx_plan_host_sync(hpx_plan plan) {
  if (!plan) {
    set_error("null plan");
    return HPX_ERR_INVALID;
  }
  DeviceGuard g(plan->device);
  if (plan->aio_streams) {
    cudaStream_t* st = static_cast<cudaStream_t*>(plan->aio_streams);
    for (int i = 0; i < 2; ++i) {
      cudaError_t e = cudaStreamSynchronize(st[i]);
      if (e != cudaSuccess) return cuda_fail(e, "hpx_plan_host_sync");
    }
  }
  return read_status(plan);
}

hpx_status hpx_map2alm_host(hpx_plan plan, const void* host_map, void* host_alm, hpx_stream_t stream) {
  return host_call(plan, host_map, host_alm, stream, true);
}

hpx_status hpx_alm2map_host(hpx_plan plan, const void* host_alm, void* host_map, hpx_stream_t stream) {
  return host_call(plan, host_alm, host_map, stream, false);
}

hpx_status hpx_plan_ring_table(hpx_plan plan, int64_t* start, int32_t* nphi, double* z, double* sinth,
                               int32_t* sigma) {
  if (!plan || !start || !nphi || !z || !sinth || !sigma) {
    set_error("null argument");
    return HPX_ERR_INVALID;
  }
  DeviceGuard g(plan->device);
  std::vector<RingInfo> h(plan->nring);
  cudaError_t e = cudaMemcpy(h.data(), plan->d_ring, sizeof(RingInfo) * plan->nring, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "ring table copy");
  for (int y = 0; y < plan->nring; ++y) {
    start[y] = h[y].start;
    nphi[y] = h[y].nphi;
    z[y] = h[y].z;
    sinth[y] = h[y].sinth;
    sigma[y] = h[y].sigma;
  }
  return HPX_OK;
}

hpx_status hpx_plan_set_timing(hpx_plan plan, int enable) {
  if (!plan) {
    set_error("null plan");
    return HPX_ERR_INVALID;
  }
  if (!plan->timing) plan->timing = new TimingState();
  static_cast<TimingState*>(plan->timing)->on = enable != 0;
  return HPX_OK;
}

hpx_status hpx_plan_stage_times(hpx_plan plan, double* ms, int64_t* launches) {
  if (!plan) {
    set_error("null plan");
    return HPX_ERR_INVALID;
  }
  if (ms)
    for (int k = 0; k < kStages; ++k) ms[k] = 0.0;
  if (launches)
    for (int k = 0; k < kStages; ++k) launches[k] = 0;
  TimingState* ts = static_cast<TimingState*>(plan->timing);
  if (!ts) return HPX_OK;
  DeviceGuard g(plan->device);
  cudaError_t first = cudaSuccess;
  for (auto& r : ts->recs) {
    float t = 0.0f;
    cudaError_t e = cudaEventSynchronize(r.b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, r.a, r.b);
    if (e != cudaSuccess && first == cudaSuccess) first = e;
    if (ms) ms[r.stage] += t;
    if (launches) launches[r.stage] += r.n;
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  ts->recs.clear();
  if (first != cudaSuccess) return cuda_fail(first, "hpx_plan_stage_times");
  return HPX_OK;
}

hpx_status hpx_plan_chain_stats(hpx_plan plan, int64_t* active, int64_t* total) {
  if (!plan || !active || !total) {
    set_error("null argument");
    return HPX_ERR_INVALID;
  }
  DeviceGuard g(plan->device);
  const size_t nchain = (size_t)(plan->mmax + 1) * plan->npair;
  std::vector<int> lc(nchain);
  cudaError_t e = cudaMemcpy(lc.data(), plan->d_lc, sizeof(int) * nchain, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "chain table copy");
  long long a = 0;
  for (size_t c = 0; c < nchain; ++c)
    if (lc[c] <= plan->lmax) a += plan->lmax + 1 - lc[c];
  *active = a;
  *total = plan->nalm * (long long)plan->npair;
  return HPX_OK;
}

}  // extern "C"
