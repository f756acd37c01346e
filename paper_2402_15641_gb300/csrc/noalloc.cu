// Forward and adjoint transforms for callers that cannot allocate device
// memory.
//
// srt_forward needs a caller-provided device workspace for the intermediates
// of the two stages.  Some callers have no way to provide one: code running
// under a memory manager that owns every device allocation and forbids direct
// cudaMalloc/cudaFree, plug-ins and callbacks that are not allowed to allocate,
// or latency-critical loops where an allocation (which may synchronise the
// device) is not acceptable.  srt_forward_noalloc serves them with scratch that
// the library owns: a fixed-size array in device memory, reserved when the
// library's device code is loaded on a GPU and held until the process exits.
//
// The array is shared by every call on a device and keeps whatever the last
// call left in it.  Nothing in it has to start at zero: the transform writes
// every intermediate element before reading it.  Two calls whose work overlaps
// on the GPU (different streams, or host threads racing) use the same scratch
// and corrupt each other's results; callers must order such calls.
#include <mutex>

#include "common.cuh"

namespace {

// Scratch for srt_forward_noalloc / srt_adjoint_noalloc
// (SRT_NOALLOC_WORKSPACE_BYTES per GPU).
static __device__ __align__(256) unsigned char g_noalloc_scratch[SRT_NOALLOC_WORKSPACE_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  Host code only
// sees a host-side stand-in for g_noalloc_scratch; the device address has to
// be looked up once per device, with that device current.
int scratch_on_current_device(void** out) {
  int dev = 0;
  SRT_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return SRT_ERR_ARG;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return SRT_ERR_CUDA;
    }
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return SRT_OK;
}

// The scratch of the current device for a call of `batch` volumes on `plan`.
int noalloc_scratch(srt_plan_t plan, int32_t batch, void** scratch) {
  int dev = -1;
  SRT_CUDA_TRY(cudaGetDevice(&dev));
  if (dev != plan->device) return SRT_ERR_ARG;  // the plan lives on another GPU
  size_t need = 0;
  SRT_TRY(srt_workspace_bytes(plan, batch, &need));
  if (need > (size_t)SRT_NOALLOC_WORKSPACE_BYTES) return SRT_ERR_WORKSPACE;
  return scratch_on_current_device(scratch);
}

}  // namespace

extern "C" int srt_forward_noalloc(srt_plan_t plan, const float* f, float* p, int32_t batch,
                                   void* stream) {
  if (!plan || !f || !p || batch <= 0) return SRT_ERR_ARG;
  void* scratch = nullptr;
  SRT_TRY(noalloc_scratch(plan, batch, &scratch));
  return srt_forward(plan, f, p, batch, scratch, (size_t)SRT_NOALLOC_WORKSPACE_BYTES, stream);
}

extern "C" int srt_adjoint_noalloc(srt_plan_t plan, const float* p, float* f, int32_t batch,
                                   void* stream) {
  if (!plan || !p || !f || batch <= 0) return SRT_ERR_ARG;
  void* scratch = nullptr;
  SRT_TRY(noalloc_scratch(plan, batch, &scratch));
  return srt_adjoint(plan, p, f, batch, scratch, (size_t)SRT_NOALLOC_WORKSPACE_BYTES, stream);
}
