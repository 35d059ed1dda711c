// noalloc.cu -- emu_dgemm_noalloc: the Scheme I DGEMM with its scratch in a
// fixed, file-scope device array instead of allocated workspace.
//
// Some callers cannot allocate device memory during a call: applications
// whose device memory is already reserved up front by their own pool (a
// cudaMalloc would fail or fragment that pool), code that must not pay the
// implicit synchronisation and driver-lock cost of cudaMalloc/cudaFree on a
// latency-critical path, and plugins that run inside a host program that
// forbids them to allocate.  This entry point serves them: it calls no
// cudaMalloc, cudaFree or other allocating routine.  Its scratch (exponent
// scan results, exponents and the interleaved slices of both operands) lives
// in `g_scratch` below, which every GPU that loads the library holds until
// the process exits.
//
// The array's name is only a host-side stand-in for the device object, so
// host code obtains the real device address with cudaGetSymbolAddress, with
// the device current, the first time this entry point runs in a CUDA context
// of that device.  The address is cached per device together with the
// context's unique ID and looked up again whenever the current context's ID
// differs (after cudaDeviceReset the primary context, and with it the
// array, is created anew at another address).  Every call shares the array
// and it keeps the last call's contents; whatever must start at zero is
// cleared by each call.  Two calls whose work overlaps on the GPU (different
// streams, not ordered) race on the array.
#include <mutex>

#include "emu_handle.h"
#include "emu_internal.h"

namespace emu {
namespace {

constexpr size_t kScratchBytes = static_cast<size_t>(EMU_NOALLOC_SCRATCH_BYTES);
constexpr int kMaxDevices = 64;

static __device__ __align__(256) uint8_t g_scratch[kScratchBytes];

// Driver entry points for the current context and its unique ID (CUDA 12.0+).
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

struct DriverFns {
  CtxGetCurrentFn get_current = nullptr;
  CtxGetIdFn get_id = nullptr;
};

const DriverFns& driver_fns() {
  static DriverFns f;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      f.get_current = reinterpret_cast<CtxGetCurrentFn>(p);
    p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      f.get_id = reinterpret_cast<CtxGetIdFn>(p);
  });
  return f;
}

// Unique ID of the current context (false if there is none yet).
bool current_ctx_id(unsigned long long* id) {
  const DriverFns& f = driver_fns();
  if (!f.get_current || !f.get_id) return false;
  CUcontext ctx = nullptr;
  if (f.get_current(&ctx) != CUDA_SUCCESS || ctx == nullptr) return false;
  return f.get_id(ctx, id) == CUDA_SUCCESS;
}

struct DeviceSlot {
  bool ready = false;
  unsigned long long ctx_id = 0;
  uint8_t* addr = nullptr;
  int num_sms = 0;
};
std::mutex g_mu;
DeviceSlot g_slots[kMaxDevices];

// Set-up for the current device and context: device address of g_scratch
// and SM count.
emu_status_t scratch_for_current_device(uint8_t** addr, int* num_sms) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return EMU_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  DeviceSlot& s = g_slots[dev];
  unsigned long long id = 0;
  const bool have_id = current_ctx_id(&id);
  if (!s.ready || !have_id || id != s.ctx_id) {
    // the runtime makes the device's primary context current here if no
    // context is current yet
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      s.ready = false;
      return EMU_ERR_CUDA;
    }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return EMU_ERR_CUDA;
    if (!current_ctx_id(&id)) return EMU_ERR_CUDA;
    s.addr = static_cast<uint8_t*>(p);
    s.num_sms = sms;
    s.ctx_id = id;
    s.ready = true;
  }
  *addr = s.addr;
  *num_sms = s.num_sms;
  return EMU_OK;
}

}  // namespace
}  // namespace emu

using namespace emu;

extern "C" emu_status_t emu_dgemm_noalloc(emu_layout_t layout, int64_t m, int64_t n, int64_t k, double alpha,
                                          const double* A, int64_t lda, const double* B, int64_t ldb,
                                          double beta, double* C, int64_t ldc, int p, int* status_dev,
                                          emu_stream_t stream) {
  if (layout != EMU_ROW_MAJOR && layout != EMU_COL_MAJOR) return EMU_ERR_INVALID_ARG;
  if (m < 0 || n < 0 || k < 0) return EMU_ERR_INVALID_ARG;
  if (p < EMU_P_MIN || p > EMU_P_MAX) return EMU_ERR_UNSUPPORTED;
  if (m > INT32_MAX / 2 || n > INT32_MAX / 2 || k > (int64_t{1} << 30)) return EMU_ERR_UNSUPPORTED;
  if (!check_lds(layout, m, n, k, lda, ldb, ldc)) return EMU_ERR_INVALID_ARG;
  if (m > 0 && n > 0 && !C) return EMU_ERR_INVALID_ARG;
  if (m > 0 && n > 0 && k > 0 && (!A || !B)) return EMU_ERR_INVALID_ARG;
  View v;
  normalize(layout, m, n, A, lda, B, ldb, &v);
  if (v.M == 0 || v.N == 0) return EMU_OK;
  if (k == 0) {  // the same kernel as emu_dgemm's k == 0 path
    launch_scale_c<double>(C, ldc, v.M, v.N, beta, static_cast<cudaStream_t>(stream));
    return cudaGetLastError() == cudaSuccess ? EMU_OK : EMU_ERR_CUDA;
  }
  // the whole workspace of this product must fit in the array
  Plan pl = plan_I(v.M, v.N, k, p);
  if (pl.bytes > kScratchBytes) return EMU_ERR_UNSUPPORTED;

  uint8_t* scratch = nullptr;
  int num_sms = 0;
  emu_status_t s = scratch_for_current_device(&scratch, &num_sms);
  if (s != EMU_OK) return s;
  // A handle on the host stack (no allocation): no workspace, no tracing;
  // device-detected errors go to the caller's status word (none if null:
  // the kernels skip the flag update then).
  emu_handle_s hs;
  cudaGetDevice(&hs.device);
  hs.num_sms = num_sms;
  hs.status = status_dev;
  hs.ws = nullptr;
  hs.ws_bytes = 0;
  hs.ws_user = true;
  return run_scheme_I<double>(&hs, v, k, p, alpha, beta, C, ldc, OUT_F64, nullptr,
                              static_cast<cudaStream_t>(stream), scratch);
}
