// noalloc.cu -- gattn_fwd_noalloc: the forward for callers that cannot
// allocate device memory.  The scratch the forward needs (per-row
// log-sum-exp and the per-tile outputs of multiply-covered rows, i.e. the
// buffer gattn_fwd calls `saved`) lives in a file-scope device array of
// GATTN_NOALLOC_SCRATCH_BYTES that the CUDA module carries; this file calls
// no cudaMalloc, cudaFree or other allocating routine.
#include <mutex>

#include "internal.cuh"

// Device copy of the scratch, one per GPU that loads this library's module,
// held until the process exits.  In host code `g_noalloc_scratch` is only a
// host-side stand-in: its device address comes from cudaGetSymbolAddress.
// Under lazy module loading (CUDA's default) the driver allocates this copy
// when the module is first used on a device, which for a file without kernels
// is the cudaGetSymbolAddress below, i.e. the first gattn_fwd_noalloc call on
// that device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[GATTN_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_ptr[kMaxDevices] = {};

// Device address of the scratch on the current device; looked up once per
// device (with that device current) and cached.  nullptr on failure.
void* scratch_on_current_device() {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) {
      // leave no sticky last-error behind for the next call of this library
      (void)cudaGetLastError();
      return nullptr;
    }
    g_ptr[dev] = p;
  }
  return g_ptr[dev];
}
}  // namespace

extern "C" gattn_status gattn_fwd_noalloc(const gattn_desc* desc, const void* q, const void* k, const void* v,
                                          void* out, gattn_stream_t stream) {
  const size_t need = gattn_saved_bytes(desc);
  if (need == 0) return GATTN_ERR_INVALID_ARG;
  if (need > (size_t)GATTN_NOALLOC_SCRATCH_BYTES) return GATTN_ERR_WORKSPACE;
  void* scratch = scratch_on_current_device();
  if (!scratch) return GATTN_ERR_CUDA;
  // Every slot the forward reads is written earlier in the same call, so the
  // previous call's contents need no clearing.
  return gattn_fwd(desc, q, k, v, out, scratch, (size_t)GATTN_NOALLOC_SCRATCH_BYTES, stream);
}
