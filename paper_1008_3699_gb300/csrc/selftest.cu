// Self-test of the bounded device-side wait that the sweeps use for their
// cross-CTA hand-offs: one warp waits on a word that nothing ever sets. The
// wait gives up after its bound (about 2 s), records the timeout in the
// handle's status word and returns; the host then reads NDIAG_ETIMEOUT and
// the handle stays usable.
#include "sweep_common.cuh"

namespace nd {
namespace {

using namespace sweep;

__global__ void selftest_wait_kernel(const unsigned* word, DevStatus* st) {
  if (threadIdx.x == 0) (void)wait_gmem(word, 1u, st);
}

}  // namespace

ndiag_status check_device_status(Handle* h);

}  // namespace nd

using namespace nd;

extern "C" ndiag_status ndiag_selftest_wait(ndiag* h) {
  if (!h) return NDIAG_EINVAL;
  unsigned* word = (unsigned*)dev_alloc(sizeof(unsigned), h->stream);
  if (!word) return NDIAG_ENOMEM;
  ndiag_status st = NDIAG_OK;
  cudaError_t e = cudaMemsetAsync(word, 0, sizeof(unsigned), h->stream);
  if (e == cudaSuccess) {
    ++h->launches;
    selftest_wait_kernel<<<1, 32, 0, h->stream>>>(word, h->status);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) st = cuda_status(e, "ndiag_selftest_wait");
  if (st == NDIAG_OK) st = check_device_status(h);  // waits for the kernel; NDIAG_ETIMEOUT expected
  dev_free(word, sizeof(unsigned), h->stream);
  return st;
}
