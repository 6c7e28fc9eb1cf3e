// Warp-synchronous wavefront for the decomposed 9-point triangular sweeps
// (fp64; the forward and backward sweeps of the ILU(0) apply), sm_103a.
//
// The sweep and its reading of the 9-point molecule are those of sweep9.cu
// (Sec. 3): inside a subdomain the cells are taken in the lexicographic order
// of the frame reflected so that the sweep runs towards +x, +y; the new values
// of a cell are its W, SW, S and SE neighbours; across an interface only face
// neighbours couple, and only where both subdomains start at it (mutual pairs
// and the 4-cell corner, solved together, Eqs. 2d:sor2b2 and 2d:sor4b4);
// diagonal neighbours across an interface are dropped from the triangular
// factors. Per cell
//        x = h - gW xW - gSW xSW - gS xS - gSE xSE,  h = r / p or r.
//
// Design (one CTA per "unit": one subdomain, or the two subdomains of a
// mutual x-interface):
// * Band warps: lane = row, 32 rows per warp, one warp per band and
//   subdomain. At step s lane l takes column s - 2l (skew 2: the SE neighbour
//   (x + 1, y - 1) is then one step older). The W value is the lane's own last
//   result; SE arrives by shuffle from lane l - 1, and S and SW are the two
//   values received before it. Lane 0 reads the row below from a shared ring
//   written by the band below (or by the edge warp), one mbarrier per group
//   of 8 columns; every row of a subdomain fits the ring, so no slot is
//   reused.
// * The x-pair of a mutual interface: lane l of band b of both subdomains
//   reaches column 0 of the same row at the same step; the two warps exchange
//   their partial sums through shared memory under a named barrier and both
//   solve the 2x2 system with the pair's 1 / (1 - g_ab g_ba), precomputed.
// * Edge warp (a y-coupled start row): the start row of each subdomain and its
//   twin row across the interface form a recurrence of 2x2 systems that
//   depends on nothing else (Eq. 2d:sor2b2 along the line), with the 4x4
//   corner block at column 0 when the unit is an x-pair. The 32 lanes prepare
//   the operands of 32 positions at a time; lane m then advances line m. The
//   unit on the other side of the interface evaluates the same systems with the
//   same operations in a canonical member order, so both agree bit for bit.
// * Operands: the scaled coefficients of the phase are copied once per
//   coefficient set into a packed order -- (unit, subdomain, band, step,
//   lane) -- with the structural zeros in place (no row below, SW across the
//   x-interface, SE at the last column), so a step's loads are coalesced and
//   the step has no predicates on coefficients. The right-hand side is read in
//   the natural layout; results leave through shared memory as row segments.
// Every wait is bounded; after a failed wait a warp keeps stepping (so the
// named barriers stay matched) and the status word reports NDIAG_ETIMEOUT.
#include <algorithm>

#include "sweep_common.cuh"

namespace nd {
namespace {

using namespace sweep;

constexpr int WCH = 4;       // steps per chunk
constexpr int WNB = 4;       // band warps per subdomain (at most)
constexpr int WGRP = 8;      // columns per hand-off group

// index 0..7 of c[] (W E S N SW SE NW NE) of the neighbour at local offset
// (dx, dy) in the frame with corner bits (cx, cy)
__host__ __device__ inline int went(int dx, int dy, int cx, int cy) {
  const int gx = cx ? -dx : dx, gy = cy ? -dy : dy;
  if (gy == 0) return gx < 0 ? 0 : 1;
  if (gx == 0) return gy < 0 ? 2 : 3;
  if (gy < 0) return gx < 0 ? 4 : 5;
  return gx < 0 ? 6 : 7;
}

struct WUnit {
  int iy, start, cnt;
};

struct WParams {
  int nx, ny;
  Split sx, sy;
  int base;       // start corner of subdomain 0 at this phase
  int pair_par;   // parity of the x index that begins an x-pair
  int units;      // units per row of subdomains
  int nbw;        // band warps per subdomain in the launch
  int nstep;      // step slots per band in the packed copy
  int wmax, hmax;
  int ngrp;       // hand-off groups per ring (ceil(wmax / WGRP))
  int64_t pks;    // slots per packed array
  const double* pk;
  const double* rdx;   // [unit][row]: 1 / (1 - g_ab g_ba) of the x-pair
  const double* inv;   // natural scaled set (edge warp)
  const double* c0;    // entries: c0 + e * N, e = 0..7
  int64_t N;
  const double* rhs;
  double* xnew;
  DevStatus* st;
};

__host__ __device__ inline WUnit unit_of(const WParams& P, int b) {
  WUnit u;
  u.iy = b / P.units;
  const int k = b % P.units;
  u.start = P.pair_par == 0 ? 2 * k : (k == 0 ? 0 : 2 * k - 1);
  u.cnt = (P.pair_par == 1 && k == 0) ? 1 : min(2, P.sx.p - u.start);
  return u;
}

// Frame of subdomain (ix, iy) at the phase of P: extent, corner bits, whether
// its start row lies on a coupled y-interface.
struct WFrame {
  int x0, y0, w, h, cx, cy, ycoup, nx;
  __host__ __device__ int64_t gi(int x, int y) const {
    const int gx = cx ? x0 + w - 1 - x : x0 + x, gy = cy ? y0 + h - 1 - y : y0 + y;
    return (int64_t)gy * nx + gx;
  }
};

__host__ __device__ inline WFrame frame_of(const WParams& P, int ix, int iy) {
  WFrame f;
  f.nx = P.nx;
  f.x0 = P.sx.lo(ix);
  f.w = P.sx.len(ix);
  f.y0 = P.sy.lo(iy);
  f.h = P.sy.len(iy);
  const int c = P.base ^ (ix & 1) ^ ((iy & 1) << 1);
  f.cx = c & 1;
  f.cy = (c >> 1) & 1;
  f.ycoup = f.cy ? (f.y0 + f.h < P.ny) : (f.y0 > 0);
  return f;
}

// Packed arrays: KIND_TRI_SCALED inv, W, SW, S, SE; KIND_TRI_UNIT W, SW, S, SE.
template <int KIND>
struct WArr {
  static constexpr int NA = KIND == KIND_TRI_SCALED ? 5 : 4;
  static constexpr int W = NA - 4, SW = NA - 3, S = NA - 2, SE = NA - 1;
};

__host__ __device__ inline int64_t wslot(const WParams& P, int unit, int m, int band, int step, int lane) {
  return ((((int64_t)unit * 2 + m) * P.nbw + band) * P.nstep + step) * 32 + lane;
}

// The packed copy of one phase: one thread per slot (zero outside the cells);
// slots of column 0 of an x-pair also write the pair's 1 / (1 - g_ab g_ba).
template <int KIND>
__global__ void w9_pack_kernel(WParams P, double* __restrict__ pk, double* __restrict__ rdx, int64_t total) {
  using AR = WArr<KIND>;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int lane = (int)(q & 31);
    int64_t r = q >> 5;
    const int step = (int)(r % P.nstep);
    r /= P.nstep;
    const int band = (int)(r % P.nbw);
    r /= P.nbw;
    const int m = (int)(r & 1);
    const int unit = (int)(r >> 1);
    double v[AR::NA];
#pragma unroll
    for (int a = 0; a < AR::NA; ++a) v[a] = 0.0;
    const WUnit U = unit_of(P, unit);
    if (m < U.cnt) {
      const WFrame F = frame_of(P, U.start + m, U.iy);
      const int rows_b = min(32, F.h - F.ycoup - 32 * band);
      const int y = F.ycoup + 32 * band + lane, x = step - 2 * lane;
      if (lane < rows_b && x >= 0 && x < F.w) {
        const int64_t gi = F.gi(x, y);
        if (KIND == KIND_TRI_SCALED) v[0] = P.inv[gi];
        v[AR::W] = P.c0[went(-1, 0, F.cx, F.cy) * P.N + gi];
        if (y > 0) {
          v[AR::S] = P.c0[went(0, -1, F.cx, F.cy) * P.N + gi];
          if (x > 0) v[AR::SW] = P.c0[went(-1, -1, F.cx, F.cy) * P.N + gi];
          if (x + 1 < F.w) v[AR::SE] = P.c0[went(1, -1, F.cx, F.cy) * P.N + gi];
        }
        if (x == 0 && m == 0 && U.cnt == 2) {
          const WFrame B = frame_of(P, U.start + 1, U.iy);
          const double gab = v[AR::W];
          const double gba = P.c0[went(-1, 0, B.cx, B.cy) * P.N + B.gi(0, y)];
          rdx[(int64_t)unit * P.hmax + y] = 1.0 / fma(-gab, gba, 1.0);
        }
      }
    }
#pragma unroll
    for (int a = 0; a < AR::NA; ++a) pk[a * P.pks + q] = v[a];
  }
}

// Right-hand side term of a cell: r / p (scaled form) or r (unit form).
template <int KIND>
__device__ __forceinline__ double wh(const WParams& P, int64_t gi) {
  return KIND == KIND_TRI_SCALED ? __ldg(P.inv + gi) * __ldg(P.rhs + gi) : __ldg(P.rhs + gi);
}

struct WSmem {
  double* ring;            // [2][nbw][wmax + 2]: the row below each band
  double* xo;              // [2][nbw][32][WCH + 1]: a chunk's results
  double* xch;             // [2][nbw][32]: x-pair exchange
  double* ed;              // [2][7][32]: edge operands of 32 positions
  double* corner;          // [4]
  unsigned long long* full;  // [2][nbw][ngrp]
};

__device__ __forceinline__ WSmem wsmem(const WParams& P, unsigned char* base) {
  WSmem S;
  double* d = reinterpret_cast<double*>(base);
  S.ring = d;
  d += 2 * P.nbw * (P.wmax + 2);
  S.xo = d;
  d += 2 * P.nbw * 32 * (WCH + 1);
  S.xch = d;
  d += 2 * P.nbw * 32;
  S.ed = d;
  d += 2 * 7 * 32;
  S.corner = d;
  d += 4;
  S.full = reinterpret_cast<unsigned long long*>(d);
  return S;
}

size_t wsmem_bytes(int nbw, int wmax, int ngrp) {
  return sizeof(double) * ((size_t)2 * nbw * (wmax + 2) + (size_t)2 * nbw * 32 * (WCH + 1) + (size_t)2 * nbw * 32 +
                           2 * 7 * 32 + 4) +
         sizeof(unsigned long long) * (size_t)2 * nbw * ngrp;
}

// The 4-cell corner of an x-pair on a coupled y-interface: own cells A, B
// (column 0, row 0) and their twins A', B' across the y-interface. Faces
// couple (A-B and A'-B' through W, A-A' and B-B' through S); diagonals are
// dropped. Members are taken in ascending global index, so the unit on the
// other side of the interface builds and solves the same system. Results in
// S.corner: A, B, A', B'.
template <int KIND>
__device__ void w9_corner(const WParams& P, const WFrame* F, const WFrame* T, double* out) {
  int64_t gi[4];
  double hv[4], M[4][4];
  int eW[4], eS[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int m = q & 1;
    const WFrame& f = q < 2 ? F[m] : T[m];
    gi[q] = f.gi(0, 0);
    eW[q] = went(-1, 0, f.cx, f.cy);
    eS[q] = went(0, -1, f.cx, f.cy);
  }
  // canonical order of the members
  int ord[4] = {0, 1, 2, 3};
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 3 - a; ++b)
      if (gi[ord[b]] > gi[ord[b + 1]]) {
        const int t = ord[b];
        ord[b] = ord[b + 1];
        ord[b + 1] = t;
      }
  int pos[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) pos[ord[i]] = i;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
#pragma unroll
    for (int j = 0; j < 4; ++j) M[i][j] = i == j ? 1.0 : 0.0;
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i = pos[q];
    hv[i] = wh<KIND>(P, gi[q]);
    M[i][pos[q ^ 1]] = __ldg(P.c0 + eW[q] * P.N + gi[q]);  // x-face partner
    M[i][pos[q ^ 2]] = __ldg(P.c0 + eS[q] * P.N + gi[q]);  // y-face partner
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
#pragma unroll
    for (int i = k + 1; i < 4; ++i) {
      const double f = k == 0 ? M[i][0] : M[i][k] / M[k][k];
#pragma unroll
      for (int j = k + 1; j < 4; ++j) M[i][j] = fma(-f, M[k][j], M[i][j]);
      hv[i] = fma(-f, hv[k], hv[i]);
    }
  }
  double xs[4];
#pragma unroll
  for (int k = 3; k >= 0; --k) {
    double t = hv[k];
#pragma unroll
    for (int j = k + 1; j < 4; ++j) t = fma(-M[k][j], xs[j], t);
    xs[k] = k == 0 ? t : t / M[k][k];
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) out[q] = xs[pos[q]];
}

// Edge warp: the start rows (and their twin rows) of a unit on a coupled
// y-interface. Position x of line m is the 2x2 system
//   x_o + g_ot x_t = h_o - gW_o x_o(x - 1),  x_t + g_to x_o = h_t - gW_t x_t(x - 1)
// solved as x_o = (u_o - g_ot u_t) d, x_t = (u_t - g_to u_o) d with
// d = 1 / (1 - g_ot g_to): the same expressions with o and t swapped, so the
// twin unit's evaluation gives the same bits.
template <int KIND>
__device__ void w9_edge(const WParams& P, const WUnit& U, const WFrame* F, const WSmem& S, int lane) {
  WFrame T[2];
  const int iyt = F[0].cy ? U.iy + 1 : U.iy - 1;
  for (int m = 0; m < U.cnt; ++m) T[m] = frame_of(P, U.start + m, iyt);
  if (U.cnt == 2 && lane == 0) w9_corner<KIND>(P, F, T, S.corner);
  __syncwarp();
  const int wl = max(F[0].w, U.cnt == 2 ? F[1].w : 0);
  double xo_prev = 0.0, xt_prev = 0.0;
  for (int cb = 0; cb < wl; cb += 32) {
    const int x = cb + lane;
    for (int m = 0; m < U.cnt; ++m) {
      double* e = S.ed + m * 7 * 32 + lane;
      if (x < F[m].w) {
        const int64_t go = F[m].gi(x, 0), gt = T[m].gi(x, 0);
        const double got = __ldg(P.c0 + went(0, -1, F[m].cx, F[m].cy) * P.N + go);
        const double gto = __ldg(P.c0 + went(0, -1, T[m].cx, T[m].cy) * P.N + gt);
        e[0] = wh<KIND>(P, go);
        e[32] = wh<KIND>(P, gt);
        e[64] = x > 0 ? __ldg(P.c0 + went(-1, 0, F[m].cx, F[m].cy) * P.N + go) : 0.0;
        e[96] = x > 0 ? __ldg(P.c0 + went(-1, 0, T[m].cx, T[m].cy) * P.N + gt) : 0.0;
        e[128] = got;
        e[160] = gto;
        e[192] = 1.0 / fma(-got, gto, 1.0);
      }
    }
    __syncwarp();
    if (lane < U.cnt) {
      const int m = lane;
      const double* e = S.ed + m * 7 * 32;
      double* ring = S.ring + (size_t)m * P.nbw * (P.wmax + 2);  // band 0's input
      unsigned long long* full = S.full + (size_t)m * P.nbw * P.ngrp;
      const int hi = min(32, F[m].w - cb);
      for (int p = 0; p < hi; ++p) {
        const int xx = cb + p;
        double xo, xt;
        if (xx == 0 && U.cnt == 2) {
          xo = S.corner[m];
          xt = S.corner[2 + m];
        } else {
          const double uo = fma(-e[64 + p], xo_prev, e[p]);
          const double ut = fma(-e[96 + p], xt_prev, e[32 + p]);
          xo = fma(-e[128 + p], ut, uo) * e[192 + p];
          xt = fma(-e[160 + p], uo, ut) * e[192 + p];
        }
        ring[xx] = xo;
        P.xnew[F[m].gi(xx, 0)] = xo;
        xo_prev = xo;
        xt_prev = xt;
        if (xx % WGRP == WGRP - 1 || xx == F[m].w - 1) mb_arrive(&full[xx / WGRP]);
      }
    }
    __syncwarp();
  }
}

// Band warp b of subdomain m: rows ycoup + 32 b + lane.
template <int KIND>
__device__ void w9_band(const WParams& P, const WUnit& U, const WFrame& F, const WSmem& S, int m, int b, int lane,
                        int nb) {
  using AR = WArr<KIND>;
  constexpr int NA = AR::NA;
  const int rows_b = min(32, F.h - F.ycoup - 32 * b);
  const bool row_on = lane < rows_b;
  const int y = F.ycoup + 32 * b + (row_on ? lane : 0);
  const int64_t rowbase = F.gi(0, y);
  const int dx = F.cx ? -1 : 1;
  const bool has_below = b > 0 || F.ycoup;
  const bool out_next = b + 1 < nb;
  const bool paired = U.cnt == 2;
  const double rd = (paired && row_on) ? __ldg(P.rdx + (int64_t)blockIdx.x * P.hmax + y) : 1.0;
  const int nsteps = F.w + 2 * (rows_b - 1);
  const int nch = (nsteps + WCH - 1) / WCH;
  const double* pkb = P.pk + wslot(P, blockIdx.x, m, b, 0, lane);
  const double* ring_in = S.ring + ((size_t)m * P.nbw + b) * (P.wmax + 2);
  double* ring_out = S.ring + ((size_t)m * P.nbw + b + 1) * (P.wmax + 2);
  unsigned long long* full_in = S.full + ((size_t)m * P.nbw + b) * P.ngrp;
  unsigned long long* full_out = S.full + ((size_t)m * P.nbw + b + 1) * P.ngrp;
  double* xo = S.xo + ((size_t)m * P.nbw + b) * 32 * (WCH + 1);
  double* xch_own = S.xch + ((size_t)m * P.nbw + b) * 32;
  const double* xch_oth = S.xch + ((size_t)(m ^ 1) * P.nbw + b) * 32;
  // operands of a chunk: the packed arrays and the right-hand side
  double cur[NA + 1][WCH], nxt[NA + 1][WCH];
  auto load = [&](int k, double (&dst)[NA + 1][WCH]) {
#pragma unroll
    for (int j = 0; j < WCH; ++j) {
      const int s = k * WCH + j, x = s - 2 * lane;
      const int sc = min(s, P.nstep - 1);
#pragma unroll
      for (int a = 0; a < NA; ++a) dst[a][j] = __ldg(pkb + a * P.pks + (int64_t)sc * 32);
      dst[NA][j] = (row_on && x >= 0 && x < F.w) ? __ldg(P.rhs + rowbase + (int64_t)dx * x) : 0.0;
    }
  };
  load(0, nxt);
  bool ok = true;
  double xp = 0.0, hS = 0.0, hSW = 0.0;
  const int pair_last = 2 * (rows_b - 1);  // last step at which some lane sits at column 0
  for (int k = 0; k < nch; ++k) {
#pragma unroll
    for (int a = 0; a <= NA; ++a)
#pragma unroll
      for (int j = 0; j < WCH; ++j) cur[a][j] = nxt[a][j];
    if (k + 1 < nch) load(k + 1, nxt);
    const int s0 = k * WCH;
    if (has_below && ok && s0 < F.w) ok = mb_wait(&full_in[min(s0 + WCH, F.w - 1) / WGRP], 0, P.st);
#pragma unroll
    for (int j = 0; j < WCH; ++j) {
      const int s = s0 + j, x = s - 2 * lane;
      const double sh = __shfl_up_sync(FULL, xp, 1);
      double se;
      if (lane == 0) {
        const bool in = has_below && x >= 0 && x < F.w;
        se = (in && x + 1 < F.w) ? ring_in[x + 1] : 0.0;
        hS = in ? ring_in[x] : 0.0;
        hSW = (in && x > 0) ? ring_in[x - 1] : 0.0;
      } else {
        se = sh;
      }
      const double hterm = KIND == KIND_TRI_SCALED ? cur[0][j] * cur[NA][j] : cur[NA][j];
      const double u = fma(-cur[AR::SE][j], se, fma(-cur[AR::SW][j], hSW, fma(-cur[AR::S][j], hS, hterm)));
      double xn;
      if (paired && (s & 1) == 0 && s <= pair_last) {
        // lane s / 2 is at column 0: exchange u with the partner subdomain's warp
        if (x == 0) xch_own[lane] = u;
        asm volatile("bar.sync %0, 64;" ::"r"(1 + b) : "memory");
        const double up = xch_oth[lane];
        xn = x == 0 ? fma(-cur[AR::W][j], up, u) * rd : fma(-cur[AR::W][j], xp, u);
        asm volatile("bar.sync %0, 64;" ::"r"(1 + b) : "memory");
      } else {
        xn = fma(-cur[AR::W][j], xp, u);
      }
      hSW = hS;
      hS = se;
      xo[lane * (WCH + 1) + j] = xn;
      if (row_on && x >= 0 && x < F.w) {
        xp = xn;
        if (lane == 31 && out_next) ring_out[x] = xn;
      }
    }
    __syncwarp();
    {  // the chunk's results as row segments
      constexpr int RPI = 32 / WCH;
      const int jl = lane % WCH, rr = lane / WCH;
#pragma unroll
      for (int i = 0; i < WCH; ++i) {
        const int rl = rr + RPI * i, xc = s0 + jl - 2 * rl;
        if (rl < rows_b && xc >= 0 && xc < F.w) P.xnew[F.gi(xc, F.ycoup + 32 * b + rl)] = xo[rl * (WCH + 1) + jl];
      }
    }
    if (lane == 31 && out_next) {  // lane 31 finished columns s0 - 62 .. s0 + WCH - 63
      for (int c = max(0, s0 - 62); c <= min(F.w - 1, s0 + WCH - 63); ++c)
        if (c % WGRP == WGRP - 1 || c == F.w - 1) mb_arrive(&full_out[c / WGRP]);
    }
    __syncwarp();
  }
}

template <int KIND>
__global__ void __launch_bounds__(32 * (2 * WNB + 1)) sweep9w_kernel(WParams P) {
  extern __shared__ __align__(16) unsigned char w9sm[];
  const WSmem S = wsmem(P, w9sm);
  const WUnit U = unit_of(P, blockIdx.x);
  if (threadIdx.x == 0) {
    for (int i = 0; i < 2 * P.nbw * P.ngrp; ++i) mb_init(&S.full[i], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  WFrame F[2];
  F[0] = frame_of(P, U.start, U.iy);
  F[1] = U.cnt == 2 ? frame_of(P, U.start + 1, U.iy) : F[0];
  if (wid == 2 * P.nbw) {
    if (F[0].ycoup) w9_edge<KIND>(P, U, F, S, lane);
    return;
  }
  const int m = wid / P.nbw, b = wid % P.nbw;
  if (m >= U.cnt) return;
  const int rows = F[m].h - F[m].ycoup;
  const int nb = (rows + 31) / 32;
  if (b >= nb) return;
  w9_band<KIND>(P, U, F[m], S, m, b, lane, nb);
}

}  // namespace

// Launcher: NDIAG_EINVAL (nothing launched) when the request is outside what
// this kernel covers; the caller then runs the level kernel.
ndiag_status launch_sweep9w(Handle* h, int kind, int mode, int64_t t, const ScaledSet& set, const void* rhs,
                            void* xnew) {
  if (h->precision != NDIAG_FP64 || mode != NDIAG_DECOMPOSED || h->dim != 2 || h->stencil != 9) return NDIAG_EINVAL;
  if (kind != KIND_TRI_SCALED && kind != KIND_TRI_UNIT) return NDIAG_EINVAL;
  WParams P{};
  P.nx = (int)h->n[0];
  P.ny = (int)h->n[1];
  const int px = h->sub[0], py = h->sub[1];
  P.sx = Split{px, P.nx / px, P.nx % px};
  P.sy = Split{py, P.ny / py, P.ny % py};
  P.wmax = P.sx.len(0);
  P.hmax = P.sy.len(0);
  P.nbw = (P.hmax + 31) / 32;
  if (P.nbw > WNB) return NDIAG_EINVAL;
  P.base = base_corner(2, t);
  P.pair_par = (P.base & 1) ? 0 : 1;
  P.units = P.pair_par == 0 ? (px + 1) / 2 : 1 + px / 2;
  P.nstep = P.wmax + 62;
  P.ngrp = (P.wmax + WGRP - 1) / WGRP;
  const size_t smem = wsmem_bytes(P.nbw, P.wmax, P.ngrp);
  if (smem > 200 * 1024) return NDIAG_EINVAL;
  const int U = P.units * py;
  P.pks = (int64_t)U * 2 * P.nbw * P.nstep * 32;
  P.N = h->N;
  P.inv = (const double*)set.base;
  P.c0 = P.inv + h->N;
  P.rhs = (const double*)rhs;
  P.xnew = (double*)xnew;
  P.st = h->status;
  const int na = kind == KIND_TRI_SCALED ? 5 : 4;
  // the packed copy of this set, phase and kind (rebuilt when the set changes)
  PackCache* pc = nullptr;
  for (PackCache& c : h->w9pack)
    if (c.t == t && c.kind == kind) pc = &c;
  if (!pc) {
    h->w9pack.push_back(PackCache{});
    pc = &h->w9pack.back();
    pc->t = t;
    pc->kind = kind;
  }
  const size_t bytes = sizeof(double) * (size_t)na * (size_t)P.pks;
  const size_t rbytes = sizeof(double) * (size_t)U * P.hmax;
  if (pc->set_base != set.base || pc->set_version != set.version || pc->sub0 != px || pc->sub1 != py ||
      !pc->buf) {
    if (pc->bytes != bytes) {
      dev_free(pc->buf, pc->bytes, h->stream);
      pc->buf = (double*)dev_alloc(bytes, h->stream);
      pc->bytes = pc->buf ? bytes : 0;
    }
    if (pc->rdx_bytes != rbytes) {
      dev_free(pc->rdx, pc->rdx_bytes, h->stream);
      pc->rdx = (double*)dev_alloc(rbytes, h->stream);
      pc->rdx_bytes = pc->rdx ? rbytes : 0;
    }
    if (!pc->buf || !pc->rdx) {
      pc->set_base = nullptr;
      return NDIAG_ENOMEM;
    }
    ND_CUDA(cudaMemsetAsync(pc->rdx, 0, rbytes, h->stream));
    const int64_t total = P.pks;
    const unsigned grid = (unsigned)std::min<int64_t>((total + 255) / 256, (int64_t)h->sm_count * 16);
    ++h->launches;
    if (kind == KIND_TRI_SCALED)
      w9_pack_kernel<KIND_TRI_SCALED><<<grid, 256, 0, h->stream>>>(P, pc->buf, pc->rdx, total);
    else
      w9_pack_kernel<KIND_TRI_UNIT><<<grid, 256, 0, h->stream>>>(P, pc->buf, pc->rdx, total);
    ND_CUDA(cudaGetLastError());
    pc->set_base = set.base;
    pc->set_version = set.version;
    pc->sub0 = px;
    pc->sub1 = py;
  }
  P.pk = pc->buf;
  P.rdx = pc->rdx;
  static bool attr[2] = {false, false};
  const int ki = kind == KIND_TRI_SCALED ? 0 : 1;
  if (!attr[ki]) {
    if (kind == KIND_TRI_SCALED)
      ND_CUDA(cudaFuncSetAttribute(sweep9w_kernel<KIND_TRI_SCALED>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   200 * 1024));
    else
      ND_CUDA(cudaFuncSetAttribute(sweep9w_kernel<KIND_TRI_UNIT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   200 * 1024));
    attr[ki] = true;
  }
  // algorithmic bytes: the coefficients of the kind, the right-hand side and the result
  const double cellbytes = (kind == KIND_TRI_SCALED ? 5.0 : 4.0) * 8.0 + 2.0 * 8.0;
  const int slot = prof_begin(h);
  ++h->launches;
  ++h->sweep_launches;
  const unsigned threads = 32u * (2u * (unsigned)P.nbw + 1u);
  if (kind == KIND_TRI_SCALED)
    sweep9w_kernel<KIND_TRI_SCALED><<<(unsigned)U, threads, smem, h->stream>>>(P);
  else
    sweep9w_kernel<KIND_TRI_UNIT><<<(unsigned)U, threads, smem, h->stream>>>(P);
  ND_CUDA(cudaGetLastError());
  prof_end(h, slot, cellbytes * (double)h->N);
  return NDIAG_OK;
}

void w9pack_free(Handle* h) {
  for (PackCache& c : h->w9pack) {
    dev_free(c.buf, c.bytes, h->stream);
    dev_free(c.rdx, c.rdx_bytes, h->stream);
  }
  h->w9pack.clear();
  for (PackCache& c : h->brec3d) dev_free(c.buf, c.bytes, h->stream);
  h->brec3d.clear();
}

}  // namespace nd
