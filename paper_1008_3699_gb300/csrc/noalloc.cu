// ilu0_apply_noalloc: the ILU(0) apply without any device allocation.
//
// ilu0_apply needs scratch device memory: the intermediate vector y of
// (D~ + L_J) y = r, and, when a subdomain is taller than one slab, the slab
// hand-off words. It allocates them on first use. Some callers cannot let a
// library allocate device memory during a call: code whose device memory is
// owned by another allocator or runtime, code that must not allocate once it
// is running (fixed-footprint or real-time service loops), and code replayed
// from a recorded command stream. This variant uses one fixed array in device
// memory that every GPU loading the library holds until the process exits.
#include <mutex>

#include "internal.h"

namespace nd {
namespace {

constexpr size_t kMaxCells = size_t(1) << 20;   // NDIAG_NOALLOC_MAX_CELLS
constexpr size_t kSyncWords = size_t(1) << 16;  // slab hand-off words
constexpr size_t kVecBytes = kMaxCells * sizeof(double);
constexpr size_t kSyncBytes = kSyncWords * sizeof(unsigned);
constexpr size_t kTwinBytes = kSyncWords * sizeof(double);
constexpr int kMaxDevices = 64;

// The scratch: [y vector | hand-off words | hand-off twin values].
static __device__ __align__(256) unsigned char g_scratch[kVecBytes + kSyncBytes + kTwinBytes];

std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device. The host-side name of a
// __device__ array is only a stand-in, so the address is looked up with that
// device current. It is looked up again on every call made while `stream` is
// not capturing (so a device reset, which may move the array, is picked up);
// while it is capturing, the address found by the last such call is used.
ndiag_status scratch_address(cudaStream_t stream, void** out) {
  int dev = -1;
  ND_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("ilu0_apply_noalloc: device ordinal out of range");
    return NDIAG_EINVAL;
  }
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  ND_CUDA(cudaStreamIsCapturing(stream, &cap));
  std::lock_guard<std::mutex> lk(g_mu);
  if (cap == cudaStreamCaptureStatusNone || !g_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p) return cuda_status(e == cudaSuccess ? cudaErrorInvalidSymbol : e,
                                                   "cudaGetSymbolAddress(scratch)");
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return NDIAG_OK;
}

}  // namespace
}  // namespace nd

using namespace nd;

extern "C" ndiag_status ilu0_apply_noalloc(ndiag* h, const void* r, void* z) {
  if (!h || !r || !z) return NDIAG_EINVAL;
  if (h->ilu_mode < 0) return NDIAG_ESTATE;
  if (h->dim != 2 || h->stencil != 5) return NDIAG_EINVAL;
  if ((size_t)h->N > kMaxCells) {
    set_error("ilu0_apply_noalloc: more cells than NDIAG_NOALLOC_MAX_CELLS");
    return NDIAG_EINVAL;
  }
  void* base = nullptr;
  ND_TRY(scratch_address(h->stream, &base));
  unsigned char* b = static_cast<unsigned char*>(base);
  void* y = b;
  unsigned* sync = reinterpret_cast<unsigned*>(b + kVecBytes);
  void* twin = b + kVecBytes + kSyncBytes;
  const int64_t tf = fwd_phase(h->dim);
  // (D~ + L_J) y = r ; (D~ + U_J) z = D~ y, as in ilu0_apply
  ND_TRY(launch_tri_sweep2d_scratch(h, KIND_TRI_SCALED, h->ilu_mode, tf, h->ilu, r, y, sync, kSyncBytes, twin,
                                    kTwinBytes));
  const int back = h->ilu_mode == NDIAG_NATURAL ? (int)MODE_NATURAL_REV : h->ilu_mode;
  return launch_tri_sweep2d_scratch(h, KIND_TRI_UNIT, back, tf ^ 1, h->ilu, y, z, sync, kSyncBytes, twin,
                                    kTwinBytes);
}
