// hpx_map2alm_noalloc: the analysis transform with its intermediate ring
// spectra in a fixed, statically allocated device array instead of the
// plan's workspace.
//
// Who needs this: callers that may not allocate device memory when they
// transform -- for example a serving loop whose device memory is owned by
// another allocator or memory pool, or latency-critical code that must not
// risk the device-wide synchronisation cudaMalloc / cudaFree can cause.  The
// call allocates nothing: no cudaMalloc, no cudaFree, no allocating library
// routine.  The caller still passes the input map and the output coefficient
// buffer, and the plan (created earlier) supplies its read-only tables.
//
// Limit: nbatch * (6 nside^2 + 4 nside - 1) complex values of the plan's real
// type must fit in kScratchBytes (16 MiB), e.g. nside 256 with up to 5 FP32
// channels or nside 512 with one FP32 channel; larger requests are rejected
// with HPX_ERR_INVALID.  The array exists once per GPU on which its module has
// been loaded (see set-up) and stays allocated until the process exits.
//
// Sharing: every call on a device uses the same array, and it keeps whatever
// the last call wrote.  Nothing in it has to start at zero here: the ring
// transform writes every spectrum bin the Legendre stage then reads, within
// the same call.  Calls whose work overlaps on the GPU (different streams,
// different host threads) race on the array; the caller must order them.
//
// Set-up: the device address of the array is looked up with
// cudaGetSymbolAddress once per device and CUDA context, on the first call
// made there, with that device current, and kept for later calls.  A device
// whose context was reset (cudaDeviceReset) gets a new context and so a
// fresh lookup.  Under lazy module loading (the CUDA default) that first
// lookup also loads the module holding the array, which may allocate the
// array's memory and synchronise once: make the first call during set-up,
// outside any loop that must not allocate, and before any stream capture.
#include <cuda.h>

#include <mutex>

#include "hpx_internal.cuh"

namespace {

constexpr size_t kScratchBytes = size_t(16) << 20;
constexpr int kMaxDevices = 64;

// The scratch array itself.  In host code its name is only a stand-in, not a
// device address; kernels get the address looked up below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

struct ScratchSlot {
  void* ptr = nullptr;
  unsigned long long ctx_id = 0;  // the context the address belongs to (0: unknown)
};

std::mutex g_setup_mutex;
ScratchSlot g_scratch[kMaxDevices];

// Unique id of the current CUDA context (cuCtxGetId), or 0 if the driver
// cannot tell; with 0 the address is looked up on every call.
unsigned long long current_context_id() {
  using GetCurrent = CUresult (*)(CUcontext*);
  using GetId = CUresult (*)(CUcontext, unsigned long long*);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<GetCurrent>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<GetId>(f);
  });
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
    return 0;
  return id;
}

// Device address of the array on `device`, which must be current.
hpx_status scratch_address(int device, void** out) {
  if (device < 0 || device >= kMaxDevices) {
    hpx::set_error("hpx_map2alm_noalloc: device %d out of range", device);
    return HPX_ERR_INVALID;
  }
  const unsigned long long ctx = current_context_id();
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  ScratchSlot& slot = g_scratch[device];
  if (!slot.ptr || ctx == 0 || slot.ctx_id != ctx) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) {
      slot = ScratchSlot{};
      return hpx::cuda_fail(e, "hpx_map2alm_noalloc: cudaGetSymbolAddress");
    }
    slot.ptr = ptr;
    slot.ctx_id = ctx;
  }
  *out = slot.ptr;
  return HPX_OK;
}

}  // namespace

extern "C" hpx_status hpx_map2alm_noalloc(hpx_plan plan, const void* map, void* alm, hpx_stream_t stream) {
  if (!plan || !map || !alm) {
    hpx::set_error("hpx_map2alm_noalloc: null argument");
    return HPX_ERR_INVALID;
  }
  if ((reinterpret_cast<uintptr_t>(map) & 15u) || (reinterpret_cast<uintptr_t>(alm) & 15u)) {
    hpx::set_error("hpx_map2alm_noalloc: data pointers must be 16-byte aligned");
    return HPX_ERR_INVALID;
  }
  if (plan->dtype != HPX_F64 && plan->dtype != HPX_F32) {
    hpx::set_error("hpx_map2alm_noalloc: the 16-bit mixed-precision dtypes are not provided here; use hpx_map2alm");
    return HPX_ERR_UNSUPPORTED;
  }
  const size_t real = plan->dtype == HPX_F64 ? sizeof(double) : sizeof(float);
  const size_t need = 2 * real * (size_t)plan->nbatch * (size_t)plan->nspec;
  if (need > kScratchBytes) {
    hpx::set_error(
        "hpx_map2alm_noalloc: this plan needs %zu bytes of ring-spectrum scratch "
        "(nbatch %d, nside %d), more than the fixed %zu-byte array; use hpx_map2alm",
        need, plan->nbatch, plan->nside, kScratchBytes);
    return HPX_ERR_INVALID;
  }
  int prev = -1;
  cudaError_t de = cudaGetDevice(&prev);
  if (de != cudaSuccess) return hpx::cuda_fail(de, "hpx_map2alm_noalloc: cudaGetDevice");
  if (prev != plan->device) {
    de = cudaSetDevice(plan->device);
    if (de != cudaSuccess) return hpx::cuda_fail(de, "hpx_map2alm_noalloc: cudaSetDevice");
  }
  void* scratch = nullptr;
  hpx_status st = scratch_address(plan->device, &scratch);
  if (st == HPX_OK) {
    // Same kernels as hpx_map2alm, pointed at the static array for the spectra.
    hpx_plan_s view = *plan;
    view.d_spec = scratch;
    view.timing = nullptr;
    if (plan->tc_mode > 0) view.d_tab = nullptr;  // a 16-bit tensor-core table: recompute lambda instead
    view.d_bmax = nullptr;                         // no operand scales: the plan's own calls own them
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int nlaunch = 0;
    cudaError_t e;
    if (plan->dtype == HPX_F64) {
      e = hpx::launch_r2c<double>(&view, static_cast<const double*>(map), s);
      if (e == cudaSuccess) e = hpx::launch_analysis<double>(&view, static_cast<double*>(alm), true, 1.0, s, &nlaunch);
    } else {
      e = hpx::launch_r2c<float>(&view, static_cast<const float*>(map), s);
      if (e == cudaSuccess) e = hpx::launch_analysis<float>(&view, static_cast<float*>(alm), true, 1.0, s, &nlaunch);
    }
    if (e != cudaSuccess) st = hpx::cuda_fail(e, "hpx_map2alm_noalloc");
  }
  if (prev != plan->device) {
    de = cudaSetDevice(prev);
    if (de != cudaSuccess && st == HPX_OK) st = hpx::cuda_fail(de, "hpx_map2alm_noalloc: restoring the device");
  }
  return st;
}
