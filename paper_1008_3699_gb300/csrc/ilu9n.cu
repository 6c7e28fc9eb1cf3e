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

// Decomposed full ILU(0): the same elimination inside every subdomain, in the
// order the subdomain's forward sweep visits its cells -- lexicographic in the
// frame reflected along the axes it sweeps backwards (start corner
// base ^ (ix & 1) ^ 2 (iy & 1), the schedule of the sweep kernels). In that
// frame the local SW, S, SE, W neighbours come first, so the natural
// kernel's elimination runs on local directions; entries that leave the
// subdomain are neither used nor changed (they stay A's and the apply couples
// across interfaces as the decomposed sweep does). Lower entries are stored as
// l_ik u_kk (rounded from the multiplier), the form of the oracle's export.
// One CTA per subdomain; row i depends on rows of its own subdomain only, on
// lower local levels lx + 2 ly.
struct FullParams {
  int nx, ny;
  Split sx, sy;
  int base;
};

// library entry of local direction e (1..8: W E S N SW SE NW NE of the frame)
__device__ __forceinline__ int frame_entry(int e, int cx, int cy) {
  if (e == 0) return 0;
  int dx = (e == EW || e == ESW || e == ENW) ? -1 : (e == EE || e == ESE || e == ENE) ? 1 : 0;
  int dy = (e == ES || e == ESW || e == ESE) ? -1 : (e == EN || e == ENW || e == ENE) ? 1 : 0;
  if (cx) dx = -dx;
  if (cy) dy = -dy;
  if (dy == 0) return dx < 0 ? EW : EE;
  if (dx == 0) return dy < 0 ? ES : EN;
  if (dy < 0) return dx < 0 ? ESW : ESE;
  return dx < 0 ? ENW : ENE;
}

__global__ void __launch_bounds__(TN) ilu9_full_kernel(FullParams P, const double* __restrict__ A,
                                                        double* __restrict__ F, DevStatus* st) {
  const int64_t N = (int64_t)P.nx * P.ny;
  const int ix = (int)blockIdx.x % P.sx.p, iy = (int)blockIdx.x / P.sx.p;
  const int cidx = P.base ^ (ix & 1) ^ ((iy & 1) << 1);
  const int cx = cidx & 1, cy = (cidx >> 1) & 1;
  const int x0 = P.sx.lo(ix), w = P.sx.len(ix), y0 = P.sy.lo(iy), hgt = P.sy.len(iy);
  int g[9];
#pragma unroll
  for (int e = 0; e < 9; ++e) g[e] = frame_entry(e, cx, cy);
  // global cell of local (lx, ly), and the step of one local unit in x / y
  const int64_t sxs = cx ? -1 : 1, sys = cy ? -(int64_t)P.nx : (int64_t)P.nx;
  auto cell = [&](int lx, int ly) {
    const int gx = cx ? x0 + w - 1 - lx : x0 + lx, gy = cy ? y0 + hgt - 1 - ly : y0 + ly;
    return (int64_t)gy * P.nx + gx;
  };
  auto u = [&](int e, int64_t k) { return __ldcg(F + (size_t)g[e] * N + k); };
  const int lmax = (w - 1) + 2 * (hgt - 1);
  for (int L = 0; L <= lmax; ++L) {
    const int ylo = max(0, (L - w + 2) / 2), yhi = min(hgt - 1, L / 2);
    for (int ly = ylo + (int)threadIdx.x; ly <= yhi; ly += TN) {
      const int lx = L - 2 * ly;
      if (lx < 0 || lx >= w) continue;
      const int64_t i = cell(lx, ly);
      double a[9];
#pragma unroll
      for (int e = 0; e < 9; ++e) a[e] = A[(size_t)g[e] * N + i];
      const bool wst = lx > 0, east = lx + 1 < w, s = ly > 0, n = ly + 1 < hgt;
      double low[4] = {0.0, 0.0, 0.0, 0.0};  // l_ik u_kk of SW, S, SE, W
      if (s && wst) {  // k = SW
        const int64_t k = i - sys - sxs;
        const double uk = u(EC, k), l = __ddiv_rn(a[ESW], uk);
        low[0] = __dmul_rn(l, uk);
        a[ES] = __dsub_rn(a[ES], __dmul_rn(l, u(EE, k)));
        a[EW] = __dsub_rn(a[EW], __dmul_rn(l, u(EN, k)));
        a[EC] = __dsub_rn(a[EC], __dmul_rn(l, u(ENE, k)));
      }
      if (s) {  // k = S
        const int64_t k = i - sys;
        const double uk = u(EC, k), l = __ddiv_rn(a[ES], uk);
        low[1] = __dmul_rn(l, uk);
        if (east) a[ESE] = __dsub_rn(a[ESE], __dmul_rn(l, u(EE, k)));
        if (wst) a[EW] = __dsub_rn(a[EW], __dmul_rn(l, u(ENW, k)));
        a[EC] = __dsub_rn(a[EC], __dmul_rn(l, u(EN, k)));
        if (east) a[EE] = __dsub_rn(a[EE], __dmul_rn(l, u(ENE, k)));
      }
      if (s && east) {  // k = SE
        const int64_t k = i - sys + sxs;
        const double uk = u(EC, k), l = __ddiv_rn(a[ESE], uk);
        low[2] = __dmul_rn(l, uk);
        a[EC] = __dsub_rn(a[EC], __dmul_rn(l, u(ENW, k)));
        a[EE] = __dsub_rn(a[EE], __dmul_rn(l, u(EN, k)));
      }
      if (wst) {  // k = W
        const int64_t k = i - sxs;
        const double uk = u(EC, k), l = __ddiv_rn(a[EW], uk);
        low[3] = __dmul_rn(l, uk);
        a[EC] = __dsub_rn(a[EC], __dmul_rn(l, u(EE, k)));
        if (n) a[ENW] = __dsub_rn(a[ENW], __dmul_rn(l, u(EN, k)));
        if (n) a[EN] = __dsub_rn(a[EN], __dmul_rn(l, u(ENE, k)));
      }
      if (s && wst) a[ESW] = low[0];
      if (s) a[ES] = low[1];
      if (s && east) a[ESE] = low[2];
      if (wst) a[EW] = low[3];
      if (a[EC] == 0.0) atomicExch(&st->zero_pivot, 1);
#pragma unroll
      for (int e = 0; e < 9; ++e) F[(size_t)g[e] * N + i] = a[e];
    }
    __syncthreads();
  }
}

}  // namespace

ndiag_status launch_ilu_factor9_full(Handle* h, double* F) {
  if (h->stencil != 9 || h->dim != 2) return NDIAG_EINVAL;
  FullParams P;
  P.nx = (int)h->n[0];
  P.ny = (int)h->n[1];
  P.sx = Split{h->sub[0], P.nx / h->sub[0], P.nx % h->sub[0]};
  P.sy = Split{h->sub[1], P.ny / h->sub[1], P.ny % h->sub[1]};
  P.base = base_corner(2, fwd_phase(2));
  ++h->launches;
  ilu9_full_kernel<<<(unsigned)(h->sub[0] * h->sub[1]), TN, 0, h->stream>>>(P, h->A64, F, h->status);
  ND_CUDA(cudaGetLastError());
  return NDIAG_OK;
}

ndiag_status launch_ilu_factor9_natural(Handle* h, double* F) {
  if (h->stencil != 9 || h->dim != 2) return NDIAG_EINVAL;
  ++h->launches;
  ilu9_natural_kernel<<<1, TN, 0, h->stream>>>((int)h->n[0], (int)h->n[1], h->A64, F, h->status);
  ND_CUDA(cudaGetLastError());
  return NDIAG_OK;
}

}  // namespace nd
