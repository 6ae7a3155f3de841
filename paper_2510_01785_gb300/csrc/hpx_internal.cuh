// Internal declarations shared by the libhpx translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <string>

#include "hpx.h"

namespace hpx {

// ---------------------------------------------------------------------------
// complex helpers (float2 / double2)
// ---------------------------------------------------------------------------
template <typename T> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };
template <typename T> using C2 = typename Vec2<T>::type;

template <typename V> __host__ __device__ __forceinline__ V cmk(decltype(V::x) a, decltype(V::x) b) {
  V r; r.x = a; r.y = b; return r;
}
template <typename V> __device__ __forceinline__ V cadd(V a, V b) { return cmk<V>(a.x + b.x, a.y + b.y); }
template <typename V> __device__ __forceinline__ V csub(V a, V b) { return cmk<V>(a.x - b.x, a.y - b.y); }
template <typename V> __device__ __forceinline__ V cconj(V a) { return cmk<V>(a.x, -a.y); }
template <typename V> __device__ __forceinline__ V cmul(V a, V b) {
  return cmk<V>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename V> __device__ __forceinline__ V cscale(V a, decltype(V::x) s) { return cmk<V>(a.x * s, a.y * s); }

// ---------------------------------------------------------------------------
// plan-resident tables
// ---------------------------------------------------------------------------
// One HEALPix ring (Sec. III-A).
struct RingInfo {
  long long start;    // first pixel in RING order
  long long specoff;  // offset of its half spectrum (N/2 + 1 bins) in the spectrum workspace
  long long etab;     // offset of its table E_N[r] = exp(-i pi r / N), r in [0, 2N)
  long long btab;     // offset of its Bluestein kernel spectrum (2^logm bins), -1 if N/2 is a power of two
  int nphi;           // N_y
  int sigma;          // phi_0 = sigma pi / N_y
  int logm;           // log2 of the FFT length used for the ring
  int pad;
  double z, sinth;    // cos(theta_y), sin(theta_y)
  double w;           // quadrature weight of every pixel on the ring (4 pi / Npix)
};

}  // namespace hpx

struct hpx_plan_s {
  int nside, lmax, mmax, nbatch, dtype, device;
  unsigned flags;
  int nring, npair;
  long long npix, nalm, nspec;
  int logm_max;        // largest FFT length over the rings (log2)
  int logtw;           // log2 of the twiddle table's FFT length
  long long netab, nbtab;
  hpx::RingInfo* d_ring;
  void* d_etab;        // C2<T> per distinct ring length
  void* d_btab;        // C2<T> Bluestein kernel spectra, natural order, scaled 1/M
  void* d_chirp;       // C2<T> per cap ring i (offset i (i - 1)): exp(-pi i n^2 / H), n < H = 2i
  void* d_tw;          // C2<T> tw[j] = exp(-2 pi i j / 2^logtw), j < 2^(logtw-1)
  double* d_cmm;       // [mmax+1] lambda_mm / sin^m(theta) (sign included)
  double* d_coef_c;    // [nalm] recurrence coefficient c_l of mu_l = c_l z mu_{l-1} - mu_{l-2}
  float2* d_coef_cf;   // [nalm] c_l as a double-FP32 pair (hi, lo): the FP32 plans' recurrence
  double* d_coef_p;    // [nalm] P_l, lambda_l = P_l mu_l
  float* d_coef_pf;    // [nalm] P_l rounded to float
  int* d_lc;           // [mmax+1][npair] first significant l of chain (m, pair)
  double* d_mu0;       // [mmax+1][npair] mu_{lc-1}
  double* d_mu1;       // [mmax+1][npair] mu_{lc}
  void* d_spec;        // workspace [nbatch][nspec] C2<T>
  void* d_F;           // workspace [nbatch][nring][mmax+1] C2<T>
  void* d_io_map;      // device I/O buffers of the host-buffer entry points (lazy)
  void* d_io_alm;
  void* d_aio_map[2];  // pipelined host-buffer calls: two I/O slots (lazy)
  void* d_aio_alm[2];
  int aio_next;        // slot of the next pipelined call
  void* aio_streams;   // cudaStream_t[2]: host-to-device, device-to-host
  void* aio_events;    // cudaEvent_t[6]: uploaded[2], computed[2], slot free[2]
  void* d_it_map;      // iterative refinement: synthesis / residual map and correction (lazy)
  void* d_it_alm;
  void* timing;        // per-stage CUDA events while timing is enabled
  void* d_tab;         // plan-resident lambda table (HPX_PLAN_LAMBDA_TABLE), C2<T>'s real type
  long long* d_tab_off;  // [mmax+1][ngroup] first element of each (m, 32-pair group)
  int* d_tab_lstart;   // [mmax+1][ngroup] first l stored for the group
  int ngroup;
  long long tab_elems;
  // tensor-core Legendre stages (HPX_PLAN_TENSOR_CORES and the 16-bit dtypes)
  int tc_nn_a, tc_nn_s;  // N columns of the analysis / synthesis tiles (0: not used)
  int tc_mode;         // 0 FP32 table (3xTF32), 1 one 16-bit product, 2 16-bit x3 (hi, lo)
  int tc_fmt;          // 16-bit operand format: 0 FP16, 1 BF16
  float tc_sfac_a, tc_sfac_s;  // channel-scale bound factors of the current transform
  void* d_tab_lo;      // 16-bit x3: remainders of the row table
  void* d_gt;          // analysis operand Gt[cgroup][m][group][rows][row width] (per transform), one
                       // region per channel group of an analysis launch
  long long gt_group_elems;  // elements of one channel group's Gt region
  int gt_groups;       // channel groups Gt holds
  void* d_at;          // synthesis operand At[group][chunk][rows][row width] (per transform), one
                       // region per channel group of a synthesis launch
  long long at_group_elems;  // elements of one channel group's At region
  int at_groups;       // channel groups At holds (the plan's nbatch over channels per group)
  long long* d_achunk; // [mmax+2] first At chunk of each m
  unsigned* d_bmax;    // [2][bmax_stride] 16-bit modes: largest operand component per channel, of
                       // the analysis (spectra) and of the synthesis (alm), apart so that an
                       // analysis and a synthesis may run on the plan at the same time
  int bmax_stride;     // the plan's own nbatch (views for fewer channels keep it)
  void* d_stab;        // column lambda table: blocks of 128 pairs x (32 or 64) l
  void* d_stab_lo;     // 16-bit x3: its remainders
  long long* d_stab_off;  // [mmax+1][nptile] first element of each (m, pair tile)
  int* d_stab_lstart;  // [mmax+1][nptile] first l stored
  int nptile;
  long long stab_elems;
  alignas(64) unsigned char tm_tab[128];   // TMA descriptors
  alignas(64) unsigned char tm_tablo[128];
  alignas(64) unsigned char tm_gt[128];
  alignas(64) unsigned char tm_stab[128];
  alignas(64) unsigned char tm_stablo[128];
  alignas(64) unsigned char tm_at[128];
  // out-of-core tables (HPX_PLAN_LAMBDA_HOST): pinned host copies, streamed
  // per block of m through two device staging buffers
  void* h_tab;
  void* h_tab_lo;
  void* h_stab;
  void* h_stab_lo;
  size_t host_bytes;   // pinned host memory of the tables
  void* d_stage[2];    // each: hi part, then (x3) lo part, stage_bytes apiece
  size_t stage_bytes;
  int stage_next;      // staging buffer of the next block
  int nblk_row, nblk_col;
  int* blk_row;        // host [nblk + 1]: m boundaries of the row-table blocks
  int* blk_col;
  long long* blk_row_base;  // host [nblk + 1]: first table element of each block
  long long* blk_col_base;
  alignas(64) unsigned char tm_stage[2][128];
  alignas(64) unsigned char tm_stagelo[2][128];
  void* copy_stream;   // cudaStream_t
  void* fft_streams;   // cudaStream_t[2]: the belt-ring launches of the analysis / synthesis ring
                       // transforms, beside the cap-ring launch on the caller's stream
  void* fft_events;    // cudaEvent_t[4]: fork / join of the analysis, then of the synthesis
  void* stage_events;  // cudaEvent_t[4]: copied[2], free[2]
  int* d_status;       // device-side wait status (HPX_OK or HPX_ERR_TIMEOUT)
  int test_withhold;   // test support: tile kernels issue no copies (hpx_plan_test_withhold_copies)
  double w_max;        // largest ring weight (4 pi / Npix unless set)
  size_t bytes;
};

namespace hpx {

// Significance threshold of the recurrence chains: a chain contributes from
// the first l at which |mu_l| >= 2^-kSigExp; earlier values are below
// 2^-kSigExp (about 1.6e-60) and are dropped.
constexpr int kSigExp = 200;

// Rows (l values) per tensor-core tile of the Legendre analysis; the lambda
// table's group starts are aligned to this grid relative to m.
constexpr int kTcTile = 128;

// error reporting (thread-local message)
void set_error(const char* fmt, ...);
hpx_status cuda_fail(cudaError_t e, const char* what);

// Let `func` launch with any dynamic shared memory size the current device
// allows.  The attribute is global per function, so plans of different sizes
// (and threads launching them) must not set it to their own sizes: one plan
// could lower it below what another, still live, launches with.  The launch
// size itself decides occupancy, not this limit.
template <typename F>
cudaError_t allow_max_smem(F* func) {
  int dev = 0, maxopt = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&maxopt, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, maxopt);
  return e;
}

// A recurrence value in the contraction's type.  The float case avoids the
// double-to-float conversion instruction, which on this GPU issues to the same
// scarce FP64 pipe as the recurrence: sign, exponent and top 24 significand
// bits are moved with integer operations (rounded half up in magnitude), and
// |x| < 2^-126 becomes 0.  |x| here is far below 2^128.  Every lambda table
// and kernel converts with this one function, so their values agree bit for
// bit.
template <typename T> __device__ __forceinline__ T to_real(double x);
template <> __device__ __forceinline__ double to_real<double>(double x) { return x; }
template <> __device__ __forceinline__ float to_real<float>(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned ahi = hi & 0x7fffffffu;
  unsigned f = __funnelshift_l(lo, ahi, 3) + 0x40000000u + ((lo >> 28) & 1u);
  f = (ahi < (897u << 20)) ? 0u : (f | (hi & 0x80000000u));
  return __uint_as_float(f);
}

// Double-FP32 numbers (Dekker's double-length arithmetic, 1971): a value is
// the unevaluated sum hi + lo of two floats, about 48 significant bits, and
// the arithmetic runs on the FP32 pipe, 64 times the FP64 pipe's rate on
// this part.  The FP32 plans run the recurrence in it: mu scaled by 2^104
// (chain starts are at least 2^-200 and |mu| stays below 2^8, so both
// parts stay normal floats; a power of two scales the linear recurrence
// exactly).  Explicitly rounded operations keep the compiler from fusing the
// error terms away.
struct Df {
  float hi, lo;
};
constexpr double kDfUp = 0x1p104;
__device__ __forceinline__ Df df_of(double x) {
  const float h = __double2float_rn(x);
  return Df{h, __double2float_rn(x - (double)h)};
}
// a b as an unnormalised pair: the rounded product, plus its rounding error
// (one FMA) and the cross terms (the lo lo term, below 2^-44 ab, dropped)
__device__ __forceinline__ Df df_mul(Df a, Df b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  return Df{p, __fmaf_rn(a.lo, b.hi, e)};
}
// t n1 - n2, renormalised: Knuth's TwoSum of the leading parts, the error
// terms added, then Dekker's FastTwoSum
__device__ __forceinline__ Df df_step(Df t, Df n1, Df n2) {
  const Df q = df_mul(t, n1);
  const float s = __fsub_rn(q.hi, n2.hi);
  const float v = __fsub_rn(s, q.hi);
  const float err = __fadd_rn(__fsub_rn(q.hi, __fsub_rn(s, v)), __fsub_rn(-n2.hi, v));
  const float f = __fadd_rn(err, __fsub_rn(q.lo, n2.lo));
  const float h = __fadd_rn(s, f);
  return Df{h, __fsub_rn(f, __fsub_rn(h, s))};
}
// the float value of a scaled pair: hi 2^-104, and 0 below 2^-126 (as to_real)
__device__ __forceinline__ float df_real(Df x) { return fabsf(x.hi) < 0x1p-22f ? 0.f : __fmul_rn(x.hi, 0x1p-104f); }

// One recurrence chain mu_l = c_l z mu_{l-1} - mu_{l-2} of a plan with real
// type T, restarted at its first significant l (lc) with the stored
// (mu_{lc-1}, mu_lc) and zero before: FP64 for FP64 plans, double-FP32 for
// the others (whose results need FP32 accuracy; the pair's ~2^-46 error per
// step stays far below it over any chain).  C is the coefficient type the
// kernels stage (8 bytes either way).  step() returns mu_l as a T; every
// kernel and table of a plan steps with it, so their values agree bit for
// bit.
template <typename T> struct Recur;
template <> struct Recur<double> {
  using C = double;
  double z = 0.0, s0 = 0.0, s1 = 0.0, n1 = 0.0, n2 = 0.0;
  __device__ __forceinline__ void start(double z_, double s0_, double s1_) {
    z = z_;
    s0 = s0_;
    s1 = s1_;
  }
  __device__ __forceinline__ double step(C c, int l, int lc) {
    double mu = fma(c * z, n1, -n2);
    if (l == lc) {
      mu = s1;
      n1 = s0;
    }
    n2 = n1;
    n1 = mu;
    return mu;
  }
};
template <> struct Recur<float> {
  using C = float2;
  Df z{0.f, 0.f}, s0{0.f, 0.f}, s1{0.f, 0.f}, n1{0.f, 0.f}, n2{0.f, 0.f};
  __device__ __forceinline__ void start(double z_, double s0_, double s1_) {
    z = df_of(z_);
    s0 = df_of(s0_ * kDfUp);
    s1 = df_of(s1_ * kDfUp);
  }
  __device__ __forceinline__ float step(C c, int l, int lc) {
    Df mu = df_step(df_mul(Df{c.x, c.y}, z), n1, n2);
    if (l == lc) {
      mu = s1;
      n1 = s0;
    }
    n2 = n1;
    n1 = mu;
    return df_real(mu);
  }
};
template <typename T> using RecCoef = typename Recur<T>::C;
// the plan's coefficients in the form Recur<T> stages
template <typename T> inline const RecCoef<T>* rec_coefs(const hpx_plan_s* p) {
  return reinterpret_cast<const RecCoef<T>*>(sizeof(T) == 4 ? (const void*)p->d_coef_cf : (const void*)p->d_coef_c);
}

__host__ __device__ inline long long alm_base(int lmax, int m) {  // index(l = 0, m); index(l, m) = alm_base + l
  return (long long)m * (2 * lmax + 1 - m) / 2;
}

// launchers (defined in hpx_fft.cu / hpx_legendre.cu)
template <typename T>
cudaError_t launch_r2c(const hpx_plan_s* p, const T* map, cudaStream_t s);
template <typename T>
cudaError_t launch_c2r(const hpx_plan_s* p, T* map, bool scale_by_weight, cudaStream_t s);
// mfac multiplies every coefficient with m > 0 on its way out (analysis) or
// in (synthesis): 1 for the transforms, 2 and 1/2 for the gradients.
template <typename T>
cudaError_t launch_analysis(const hpx_plan_s* p, T* alm, bool use_weight, double mfac, cudaStream_t s,
                            int* nlaunch);
template <typename T>
cudaError_t launch_synthesis(const hpx_plan_s* p, const T* alm, double mfac, cudaStream_t s, int* nlaunch);

// plan-time table builders (hpx_fft.cu, hpx_legendre.cu)
template <typename T>
cudaError_t build_fft_tables(hpx_plan_s* p, cudaStream_t s);
cudaError_t build_recurrence_tables(hpx_plan_s* p, cudaStream_t s);
template <typename T>
cudaError_t build_lambda_table(hpx_plan_s* p, cudaStream_t s);

// tensor-core Legendre stages (hpx_tc.cu): plan-time column table, operand
// buffers and TMA descriptors; per launch of up to tc_channels_per_launch
// channels from b0, an operand pack and then the tile kernel.  The analysis
// pack reads the ring spectra and the tile kernel writes alm; the synthesis
// pack reads alm and the tile kernel writes the ring workspace d_F.  Both
// stages pack every channel group of the transform (launch_pack_tc /
// launch_pack_at_tc per group, into the group's Gt / At region) and then run
// one tile launch over all of them (launch_tile_tc / launch_synthesis_tc with
// nb up to the plan's nbatch).
// The 16-bit dtypes (HPX_F32_BF16 ...) have only this path; their tables
// (row and column, hi and for x3 lo parts) are built here too.
int tc_columns(int nbatch, int cap);  // N of a tile for nbatch channels, at most cap per launch
int tc_mode_of(int dtype, unsigned flags);  // 0 3xTF32, 1 one 16-bit product, 2 16-bit x3; -1 none
size_t tc_extra_bytes_estimate(int nside, int lmax, int mmax, int nbatch, int mode, bool host_tables);
cudaError_t build_tc(hpx_plan_s* p, cudaStream_t s);
int tc_channels_per_launch(const hpx_plan_s* p, bool synthesis);
cudaError_t launch_pack_tc(hpx_plan_s* p, int b0, int nb, bool use_weight, cudaStream_t s);
cudaError_t launch_tile_tc(hpx_plan_s* p, float* alm, int b0, int nb, double mfac, cudaStream_t s);
cudaError_t launch_pack_at_tc(hpx_plan_s* p, const float* alm, int b0, int nb, double mfac, cudaStream_t s);
cudaError_t launch_synthesis_tc(hpx_plan_s* p, int b0, int nb, cudaStream_t s);
void free_tc_host(hpx_plan_s* p);  // out-of-core resources (pinned tables, stream, events)

}  // namespace hpx
