// Device helpers shared by the 2D sweep kernels: bounded waits, release /
// acquire flags, cp.async staging, and the small coupled systems of the
// decomposed sweep (Eqs. 2d:sor2b2 and 2d:sor4b4).
#pragma once
#include <cuda_fp16.h>

#include "internal.h"

namespace nd {
namespace sweep {

constexpr long long WAIT_CYCLES = 4000000000LL;  // ~2 s at 2 GHz
constexpr unsigned FULL = 0xffffffffu;

template <class T, class TC>
__device__ __forceinline__ T ldco(const TC* p) {
  return (T)__ldg(p);
}
template <>
__device__ __forceinline__ float ldco<float, __half>(const __half* p) {
  return __half2float(__ldg(p));
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Bounded wait until *p >= v (warp-uniform), sleeping between polls so that
// the waiting warp does not take issue slots from the producer. Returns false
// on timeout after recording it in the status word.
static __device__ __noinline__ bool wait_smem(const volatile int* p, int v, DevStatus* st) {
  if (*p >= v) {
    __threadfence_block();
    return true;
  }
  const long long t0 = clock64();
  while (*p < v) {
    if (clock64() - t0 > WAIT_CYCLES) {
      atomicExch(&st->timeout, 1);
      return false;
    }
    __nanosleep(20);
  }
  __threadfence_block();
  return true;
}
static __device__ __noinline__ bool wait_gmem(const unsigned* p, unsigned v, DevStatus* st) {
  if (ld_acquire(p) >= v) return true;
  const long long t0 = clock64();
  while (ld_acquire(p) < v) {
    if (clock64() - t0 > WAIT_CYCLES) {
      atomicExch(&st->timeout, 1);
      return false;
    }
    __nanosleep(40);
  }
  return true;
}

// mbarrier (shared memory, CTA scope): one arrival completes a phase. A waiter
// of the k-th completion (k = 0, 1, ...) tests parity k & 1.
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mb_init(unsigned long long* b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mb_arrive(unsigned long long* b) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.release.cta.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(b))
               : "memory");
}
__device__ __forceinline__ bool mb_try(unsigned long long* b, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for a phase of an mbarrier (the hardware suspends the thread
// between tests); records a timeout in the status word and returns false.
static __device__ __noinline__ bool mb_wait_slow(unsigned long long* b, unsigned parity, DevStatus* st) {
  const long long t0 = clock64();
  while (!mb_try(b, parity)) {
    if (clock64() - t0 > WAIT_CYCLES) {
      atomicExch(&st->timeout, 1);
      return false;
    }
  }
  return true;
}
__device__ __forceinline__ bool mb_wait(unsigned long long* b, unsigned parity, DevStatus* st) {
  return mb_try(b, parity) || mb_wait_slow(b, parity, st);
}

// Asynchronous 4- or 8-byte copy global -> shared (cp.async, L1-allocating).
template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(s), "l"(gmem), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Coupled pair x_a = h_a - g_ab x_b, x_b = h_b - g_ba x_a. Symmetric in
// (a, b), so both CTAs that solve a pair get identical bits.
template <class T>
__device__ __forceinline__ void pair_solve(T ha, T gab, T hb, T gba, T& xa, T& xb) {
  const T det = fma(-gab, gba, T(1));
  xa = fma(-gab, hb, ha) / det;
  xb = fma(-gba, ha, hb) / det;
}

// 4x4 corner system (Eq. 2d:sor4b4) in canonical slots ordered by global
// position: slot bit0 = larger x, bit1 = larger y; x neighbour of slot k is
// k^1, y neighbour k^2:  x_k = h_k - gx_k x_{k^1} - gy_k x_{k^2}.
template <class T>
__device__ __forceinline__ void corner_solve(const T h[4], const T gx[4], const T gy[4], T x[4]) {
  const T a11 = T(1) - gx[0] * gx[1] - gy[0] * gy[2];
  const T a12 = -(gx[0] * gy[1] + gy[0] * gx[2]);
  const T r1 = h[0] - gx[0] * h[1] - gy[0] * h[2];
  const T a21 = -(gx[3] * gy[2] + gy[3] * gx[1]);
  const T a22 = T(1) - gx[3] * gx[2] - gy[3] * gy[1];
  const T r2 = h[3] - gx[3] * h[2] - gy[3] * h[1];
  const T det = a11 * a22 - a12 * a21;
  x[0] = (r1 * a22 - a12 * r2) / det;
  x[3] = (a11 * r2 - a21 * r1) / det;
  x[1] = h[1] - gx[1] * x[0] - gy[1] * x[3];
  x[2] = h[2] - gx[2] * x[3] - gy[2] * x[0];
}

// One step of a coupled line (the pairs of Eq. 2d:sor2b2 along an interface),
// written as a linear recurrence in the previous pair:
//   x_a(k) = A_a + B_a x_a(k-1) + C_a x_b(k-1),
// with a the cell on one side, b its partner across the interface. beta_a,
// beta_b are the cells' explicit parts, g_ap / g_bp their couplings to the
// previous cell of their own line, g_ab / g_ba the couplings across. Calling
// it with (a, b) swapped gives the partner's coefficients with the same
// operations, so the two CTAs that own the two sides agree bit for bit.
__device__ __forceinline__ double rcp_rn(double x) { return __drcp_rn(x); }
__device__ __forceinline__ float rcp_rn(float x) { return __frcp_rn(x); }

template <class T>
__device__ __forceinline__ void line_coefs(T beta_a, T beta_b, T g_ap, T g_bp, T g_ab, T g_ba, T& A, T& B,
                                           T& C) {
  const T det = fma(-g_ab, g_ba, T(1));
  const T inv = rcp_rn(det);  // correctly rounded: identical in every CTA
  A = fma(-g_ab, beta_b, beta_a) * inv;
  B = -g_ap * inv;
  C = (g_ab * g_bp) * inv;
}

}  // namespace sweep
}  // namespace nd
