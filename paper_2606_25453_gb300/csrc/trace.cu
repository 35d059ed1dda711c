// trace.cu -- per-phase device timing and kernel-launch counting.
//
// When tracing is on, each phase of a call (scan, split, fused GEMM, other)
// is bracketed by two CUDA events recorded on the call's stream; reading the
// trace synchronises the events and sums their elapsed times.  Events are
// pooled and reused.  Whether tracing is on or not, the host-side launches
// of each phase sit in an NVTX range (emu.scan, emu.split, emu.gemm,
// emu.other), so that a profiler can select a phase's kernels by range;
// without a profiler attached the ranges cost a few nanoseconds.
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "emu_handle.h"

namespace emu {

namespace {
struct Mark {
  int phase;
  cudaEvent_t a, b;
};
struct Trace {
  std::vector<cudaEvent_t> pool;
  std::vector<Mark> marks;
  cudaEvent_t open[4] = {nullptr, nullptr, nullptr, nullptr};
  int64_t gemm_launches = 0, kernel_launches = 0;
  cudaEvent_t get() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
};
const char* const kPhaseName[4] = {"emu.scan", "emu.split", "emu.gemm", "emu.other"};
bool capturing(cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(st, &cs);
  return cs != cudaStreamCaptureStatusNone;
}
}  // namespace

void trace_begin(emu_handle_s* h, int phase, cudaStream_t st) {
  nvtxRangePushA(kPhaseName[phase]);
  auto* t = static_cast<Trace*>(h->trace);
  if (!t || capturing(st)) return;
  cudaEvent_t e = t->get();
  cudaEventRecord(e, st);
  t->open[phase] = e;
}

void trace_end(emu_handle_s* h, int phase, cudaStream_t st, int kernels) {
  nvtxRangePop();
  auto* t = static_cast<Trace*>(h->trace);
  if (!t) return;
  t->kernel_launches += kernels;
  if (phase == PH_GEMM) t->gemm_launches += 1;
  if (capturing(st) || !t->open[phase]) return;
  cudaEvent_t e = t->get();
  cudaEventRecord(e, st);
  t->marks.push_back({phase, t->open[phase], e});
  t->open[phase] = nullptr;
}

void trace_release(emu_handle_s* h) {
  auto* t = static_cast<Trace*>(h->trace);
  if (!t) return;
  for (auto& m : t->marks) {
    cudaEventDestroy(m.a);
    cudaEventDestroy(m.b);
  }
  for (auto e : t->pool) cudaEventDestroy(e);
  for (auto e : t->open)
    if (e) cudaEventDestroy(e);
  delete t;
  h->trace = nullptr;
}

}  // namespace emu

using namespace emu;

extern "C" {

emu_status_t emu_trace_enable(emu_handle_t h, int enable) {
  if (!h) return EMU_ERR_INVALID_ARG;
  cudaSetDevice(h->device);
  if (enable && !h->trace) h->trace = new Trace();
  if (!enable && h->trace) {
    cudaDeviceSynchronize();
    trace_release(h);
  }
  return EMU_OK;
}

emu_status_t emu_trace_read(emu_handle_t h, double* ms, int64_t* gemm_launches, int64_t* kernel_launches) {
  if (!h || !ms) return EMU_ERR_INVALID_ARG;
  for (int i = 0; i < 4; ++i) ms[i] = 0.0;
  auto* t = static_cast<Trace*>(h->trace);
  if (!t) {
    if (gemm_launches) *gemm_launches = 0;
    if (kernel_launches) *kernel_launches = 0;
    return EMU_OK;
  }
  cudaSetDevice(h->device);
  emu_status_t rc = EMU_OK;
  for (auto& m : t->marks) {
    float f = 0.f;
    if (cudaEventSynchronize(m.b) != cudaSuccess || cudaEventElapsedTime(&f, m.a, m.b) != cudaSuccess)
      rc = EMU_ERR_CUDA;
    ms[m.phase] += f;
    t->pool.push_back(m.a);
    t->pool.push_back(m.b);
  }
  t->marks.clear();
  if (gemm_launches) *gemm_launches = t->gemm_launches;
  if (kernel_launches) *kernel_launches = t->kernel_launches;
  t->gemm_launches = t->kernel_launches = 0;
  return rc;
}

}  // extern "C"
