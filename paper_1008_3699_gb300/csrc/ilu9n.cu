// Natural-order ILU(0) of a 2D 9-point matrix (the comparator of the
// decomposed factor; Sec. 5 names ILU(0) of an n-diagonal matrix, and on the
// 9-point molecule it is no longer a Gauss-Seidel pass of A, so the
// off-diagonal entries are modified as well).
//
// IKJ elimination restricted to the 9-point pattern (Saad, Iterative Methods
// for Sparse Linear Systems, Alg. 10.4), rows in natural order (x fastest).
// Row i = (x, y) eliminates its lower entries in column order SW, S, SE, W;
// for each such k, l_ik = a_ik / u_kk and, for every later entry j of row i
// that row k also holds, a_ij -= l_ik u_kj:
//     k = SW: S (E of k), W (N of k), C (NE of k)
//     k = S : SE (E of k), W (NW of k), C (N of k), E (NE of k)
//     k = SE: C (NW of k), E (N of k)
//     k = W : C (E of k), NW (N of k), N (NE of k)
// Every operation is rounded on its own, in that order.
//
// The factor is written in the form the sweep kernels apply,
//     M = L U = (D + L') D^-1 (D + U'),  D = diag(u_ii),
// L' = the eliminated lower entries before the division (l_ij u_jj) and
// U' = the upper entries u_ij, as a 9 x N matrix in the library's diagonal
// order; its scaled set (entries / u_ii, 1 / u_ii) then drives the natural
// forward and reversed sweeps of the ILU(0) apply.
//
// Row i depends on rows SW, S, SE, W: on level x + 2y they all lie below, so
// one CTA walks the levels with a barrier between them.
#include "internal.h"

namespace nd {
namespace {

constexpr int TN = 1024;

__global__ void __launch_bounds__(TN) ilu9_natural_kernel(int nx, int ny, const double* __restrict__ A,
                                                           double* __restrict__ F, DevStatus* st) {
  const int64_t N = (int64_t)nx * ny;
  const int lmax = (nx - 1) + 2 * (ny - 1);
  auto u = [&](int e, int64_t k) { return __ldcg(F + (size_t)e * N + k); };
  for (int L = 0; L <= lmax; ++L) {
    const int ylo = max(0, (L - nx + 2) / 2), yhi = min(ny - 1, L / 2);
    for (int y = ylo + (int)threadIdx.x; y <= yhi; y += TN) {
      const int x = L - 2 * y;
      if (x < 0 || x >= nx) continue;
      const int64_t i = (int64_t)y * nx + x;
      double a[9];
#pragma unroll
      for (int e = 0; e < 9; ++e) a[e] = A[(size_t)e * N + i];
      const bool w = x > 0, east = x + 1 < nx, s = y > 0, n = y + 1 < ny;
      if (s && w) {  // k = SW
        const int64_t k = i - nx - 1;
        const double l = __ddiv_rn(a[ESW], u(EC, k));
        a[ES] = __dsub_rn(a[ES], __dmul_rn(l, u(EE, k)));
        a[EW] = __dsub_rn(a[EW], __dmul_rn(l, u(EN, k)));
        a[EC] = __dsub_rn(a[EC], __dmul_rn(l, u(ENE, k)));
      }
      if (s) {  // k = S
        const int64_t k = i - nx;
        const double l = __ddiv_rn(a[ES], u(EC, k));
        if (east) a[ESE] = __dsub_rn(a[ESE], __dmul_rn(l, u(EE, k)));
        if (w) a[EW] = __dsub_rn(a[EW], __dmul_rn(l, u(ENW, k)));
        a[EC] = __dsub_rn(a[EC], __dmul_rn(l, u(EN, k)));
        if (east) a[EE] = __dsub_rn(a[EE], __dmul_rn(l, u(ENE, k)));
      }
      if (s && east) {  // k = SE
        const int64_t k = i - nx + 1;
        const double l = __ddiv_rn(a[ESE], u(EC, k));
        a[EC] = __dsub_rn(a[EC], __dmul_rn(l, u(ENW, k)));
        a[EE] = __dsub_rn(a[EE], __dmul_rn(l, u(EN, k)));
      }
      if (w) {  // k = W
        const int64_t k = i - 1;
        const double l = __ddiv_rn(a[EW], u(EC, k));
        a[EC] = __dsub_rn(a[EC], __dmul_rn(l, u(EE, k)));
        if (n) a[ENW] = __dsub_rn(a[ENW], __dmul_rn(l, u(EN, k)));
        if (n) a[EN] = __dsub_rn(a[EN], __dmul_rn(l, u(ENE, k)));
      }
      if (a[EC] == 0.0) atomicExch(&st->zero_pivot, 1);
#pragma unroll
      for (int e = 0; e < 9; ++e) F[(size_t)e * N + i] = a[e];
    }
    __syncthreads();
  }
}

}  // namespace

ndiag_status launch_ilu_factor9_natural(Handle* h, double* F) {
  if (h->stencil != 9 || h->dim != 2) return NDIAG_EINVAL;
  ++h->launches;
  ilu9_natural_kernel<<<1, TN, 0, h->stream>>>((int)h->n[0], (int)h->n[1], h->A64, F, h->status);
  ND_CUDA(cudaGetLastError());
  return NDIAG_OK;
}

}  // namespace nd
