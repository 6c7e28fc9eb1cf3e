// Decomposed sequential sweep on 2D 5-point matrices, staged version
// (sm_103a): the sweep and the coupled start lines run in separate warps.
//
// One sweep of phase t solves (Delta + L_J) x = g row by row in the order of
// the paper's multi-frontal sweep (Eqs. sor2d_sw..sor2d_nw; coupled start
// nodes by Eqs. 2d:sor4b4 and 2d:sor2b2), per cell
//        x_i = beta_i - sum_{j in J_i} gamma_ij x_j .
//
// A CTA holds one slab (up to NW bands of 32 rows) of one subdomain, in a
// local frame reflected so that the sweep runs towards +x, +y.
//
// * The coupled start lines -- the start row with the neighbour's twin row
//   (Eq. 2d:sor2b2), the start column with its twin column, and the 4x4 corner
//   (Eq. 2d:sor4b4) -- depend only on each other and on old values. Written as
//   a linear recurrence in the previous pair, x_a(k) = A + B x_a(k-1) +
//   C x_b(k-1), only A depends on the right-hand side; the pivots and B, C of
//   every position are computed once per coefficient set and phase into a line
//   table. In the sweep, one edge warp evaluates A for 32 positions at a time
//   and a second one advances the row pair and the column pair (two FMAs per
//   position), writes the start row and column and hands them to the bands.
//   The CTA on the other side of the interface evaluates the same recurrence
//   with the roles swapped and the same operations, so both sides agree bit
//   for bit without synchronising.
// * The band warps cover the rest of the slab ("band region": without the
//   coupled start row and column). Each band warp (lane = row) walks the
//   columns as a skewed wavefront: lane l handles column s - l at step s. Its
//   operands are staged into shared memory by cp.async in chunks of CH steps,
//   skewed per row (row segments of CH values, several rows per instruction);
//   shared rows have an odd pitch, so the 32 lanes' reads are conflict-free.
//   The west value is the lane's own previous result, the south value arrives
//   by shuffle (lane 0: from its input ring), and a cell costs two or three
//   FMA-pipe instructions (GB300 retires one fp64 warp instruction per 64
//   cycles per sub-partition, whatever the number of active lanes). A chunk's
//   results collect in shared memory and leave as row segments as well: a
//   store of one value per row for 32 rows is a 32-request instruction that
//   also delays every other warp's shuffles. Chunks in which every row is
//   inside the band region run without per-step predicates; the sweep
//   direction along x is a template parameter, so offsets are immediates.
// * Hand-offs inside the CTA (band to band: the top row, through a ring of
//   RING columns; edge warps to bands: start row and start column) use
//   mbarriers, one per chunk-sized group, with full and empty phases; slabs of
//   a taller subdomain (the natural ordering is one subdomain) hand over
//   through global memory and progress flags, the slabs taken in ticket order.
//   The edge chain keeps a group's values in registers and stores them after
//   the group, so no memory operation sits between two positions of its
//   recurrence. Every wait is bounded (NDIAG_ETIMEOUT).
#include <cstring>
#include <vector>

#include "sweep_common.cuh"

namespace nd {
namespace {

using namespace sweep;

constexpr int NW = 4;           // band warps per CTA
constexpr int BH = 32;          // rows per band
constexpr int SLAB = NW * BH;   // band rows per CTA
constexpr int RING = 128;       // band input ring (columns)
constexpr int NBMAX = RING / 8; // hand-off groups of a ring at the smallest group size
constexpr int NT = 7;           // line-table fields

typedef unsigned long long mbar_t;

__host__ __device__ constexpr size_t align16(size_t b) { return (b + 15) / 16 * 16; }

template <class T, class TC>
struct StagedP {
  int nx, ny;
  Split sx, sy;
  int base, spp, use_ticket, coupled, rev;
  const TC* inv;
  const TC* c[4];  // W E S N
  const T* rhs;
  const T* xold;
  T* xnew;
  T om[4];
  T bscale;
  // line table: fields inv, g_ab, g_ba, B_a, C_a, B_b, C_b; start rows indexed
  // [iy][gx] (py * nx per field), start columns [ix][gy] (px * ny per field)
  const T* rowtab;
  const T* coltab;
  int64_t rt_stride, ct_stride;
  unsigned* ticket;
  unsigned* flags;   // per slab: columns of the top row published
  unsigned* cflags;  // per slab: start-column recurrence state published
  T* chain;          // per slab: that state (2 values)
  DevStatus* st;
};

// Hand-off group (columns or rows) = one chunk of steps; one full and one
// empty barrier per group of a ring.
template <class T>
struct HandOff {
  static constexpr int ECH = sizeof(T) == 8 ? 8 : 16;
  static constexpr int NB = RING / ECH;
};

template <class T, class TC, int KIND>
struct Cfg {
  static constexpr int CH = HandOff<T>::ECH;  // steps per chunk
  static constexpr int NS = 2;                 // stages
  static constexpr int NC = KIND == KIND_SOR ? 5 : (KIND == KIND_TRI_SCALED ? 3 : 2);
  static constexpr int NV = KIND == KIND_SOR ? 2 : 1;  // rhs (+ u_old)
  static constexpr int ROWS = KIND == KIND_SOR ? BH + 1 : BH;
  static constexpr int PITCH = CH + 1;                 // odd: conflict-free
  static constexpr size_t COEF_BYTES = align16(sizeof(TC) * NS * NC * ROWS * PITCH);
  static constexpr size_t VEC_BYTES = align16(sizeof(T) * NS * NV * ROWS * PITCH);
  static constexpr size_t XO_BYTES = align16(sizeof(T) * BH * PITCH);  // results of one chunk
  static constexpr size_t WARP_BYTES = COEF_BYTES + VEC_BYTES + XO_BYTES;
  static constexpr size_t BYTES = NW * WARP_BYTES;
  static_assert(RING % CH == 0 && 32 % CH == 0, "chunks must tile the ring and the edge chunks");
};

// Implicit couplings of one cell: entries jx / jy (0 W, 1 E, 2 S, 3 N) of its
// implicit x / y neighbour, scaled by the relaxation factor.
template <class T, class TC>
__device__ __forceinline__ void cell_g(const TC* const* c, int64_t gi, int jx, int jy, bool om1, T om, T& gjx,
                                       T& gjy) {
  gjx = ldco<T, TC>(c[jx] + gi);
  gjy = ldco<T, TC>(c[jy] + gi);
  if (!om1) {
    gjx *= om;
    gjy *= om;
  }
}

// beta of one cell (direct global loads; edge warps). For SOR the opposite
// entries of jx / jy hold old values; the x term is taken before the y term so
// that every CTA evaluating a cell does the same.
template <class T, class TC, int KIND, bool OM1>
__device__ __forceinline__ T cell_beta(const StagedP<T, TC>& P, int gx, int gy, int jx, int jy, T om) {
  const int64_t gi = (int64_t)gy * P.nx + gx;
  if (KIND == KIND_SOR) {
    T acc = ldco<T, TC>(P.inv + gi) * __ldg(P.rhs + gi);
    const int ox = jx ^ 1, oy = jy ^ 1;
    const int xo = gx + (ox == 1 ? 1 : -1);
    if (xo >= 0 && xo < P.nx) acc = fma(-ldco<T, TC>(P.c[ox] + gi), __ldg(P.xold + gi + (xo - gx)), acc);
    const int yo = gy + (oy == 3 ? 1 : -1);
    if (yo >= 0 && yo < P.ny)
      acc = fma(-ldco<T, TC>(P.c[oy] + gi), __ldg(P.xold + gi + (int64_t)(yo - gy) * P.nx), acc);
    return OM1 ? acc : fma(om, acc, (T(1) - om) * __ldg(P.xold + gi));
  } else if (KIND == KIND_TRI_SCALED) {
    const T beta = ldco<T, TC>(P.inv + gi) * __ldg(P.rhs + gi);
    return OM1 ? beta : beta * P.bscale;
  } else {
    return __ldg(P.rhs + gi);
  }
}

struct Geo {
  int gx0, w, gy0, h, cx, cy;
  __host__ __device__ int gxl(int lx) const { return cx ? gx0 + w - 1 - lx : gx0 + lx; }
  __host__ __device__ int gyl(int ly) const { return cy ? gy0 + h - 1 - ly : gy0 + ly; }
};

// Geometry of subdomain (ix, iy) at the launch's phase.
template <class T, class TC>
__host__ __device__ inline Geo subdomain_geo(const StagedP<T, TC>& P, int ix, int iy, bool& tx, bool& ty) {
  Geo g;
  g.gx0 = P.sx.lo(ix);
  g.w = P.sx.len(ix);
  g.gy0 = P.sy.lo(iy);
  g.h = P.sy.len(iy);
  const int cidx = P.base ^ (ix & 1) ^ ((iy & 1) << 1);
  g.cx = cidx & 1;
  g.cy = (cidx >> 1) & 1;
  tx = P.coupled && (g.cx ? (g.gx0 + g.w < P.nx) : (g.gx0 > 0));
  ty = P.coupled && (g.cy ? (g.gy0 + g.h < P.ny) : (g.gy0 > 0));
  return g;
}

// Band region of a subdomain (local rows [rlo, rhi), columns [clo, chi)) and
// the rows of one slab.
struct Region {
  int rlo, rhi, clo, chi, W;
  int slab_r0, slab_rows;
};

// Positions handled by the edge warps of one slab: the start row (slab 0)
// from column k0, the start column over the slab's rows.
struct EdgeRange {
  bool corner, row_consumer;
  int k0, nrow, ncol, l_lo, nchunks;
};

__device__ __forceinline__ EdgeRange edge_range(const Region& rg, bool tx, bool ty, int j) {
  EdgeRange e;
  e.corner = tx && ty && j == 0;
  e.k0 = e.corner ? 1 : 0;
  e.nrow = (ty && j == 0) ? max(rg.W, 0) : 0;
  e.ncol = tx ? rg.slab_rows : 0;
  e.l_lo = rg.slab_r0;
  e.row_consumer = rg.rhi > rg.rlo && rg.W > 0;
  e.nchunks = (max(e.nrow, e.ncol) + 31) / 32;
  return e;
}

// Edge warp 1 ("pre"): for 32 positions of each coupled start line at a time,
// all lanes evaluate A of both sides (B, C and the pivot come from the line
// table) into a ring of PRE slots in shared memory. All loads of a chunk are
// issued before any arithmetic (absent lines read a valid stand-in cell).
constexpr int PRE = 3;  // pre-computed position chunks in flight

template <class T, class TC, int KIND, bool OM1>
__device__ __forceinline__ void edge_pre(const StagedP<T, TC>& P, const Geo& g, int ix, int iy, const EdgeRange& er,
                                         T (*ecoef)[2][6][32], mbar_t* prefull, mbar_t* preempty, int lane) {
  const int lW = g.cx ? 1 : 0, lE = lW ^ 1, lS = g.cy ? 3 : 2, lN = lS ^ 1;
  const int cidx = g.cx | (g.cy << 1);
  const T om_p = P.om[cidx], om_q = P.om[cidx ^ 2], om_r = P.om[cidx ^ 1];
  const bool do_r = er.nrow > 0, do_c = er.ncol > 0;
  const T* rt = P.rowtab + (int64_t)iy * P.nx;
  const T* ct = P.coltab + (int64_t)ix * P.ny;
  const int64_t rs = P.rt_stride, cs = P.ct_stride;
  const int gx0c = g.gxl(0), gy0c = g.gyl(0);
  for (int c = 0; c < er.nchunks; ++c) {
    if (c >= PRE && !mb_wait(&preempty[c % PRE], ((c / PRE) - 1) & 1, P.st)) return;  // slot free again
    T(*ec)[6][32] = ecoef[c % PRE];
    const int i = 32 * c + lane;
    const int ir = min(i, max(er.nrow - 1, 0)), ic = min(i, max(er.ncol - 1, 0));
    const int gxr = do_r ? g.gxl(er.k0 + ir) : gx0c;
    const int gyq = do_r ? g.gyl(-1) : gy0c;
    const int gyc = do_c ? g.gyl(er.l_lo + ic) : gy0c;
    const int gxt = do_c ? g.gxl(-1) : gx0c;
    const T* tr = do_r ? rt + gxr : rt;
    const T* tc = do_c ? ct + gyc : ct;
    T vr[NT], vc[NT];
#pragma unroll
    for (int f = 0; f < NT; ++f) {
      vr[f] = __ldg(tr + f * rs);
      vc[f] = __ldg(tc + f * cs);
    }
    const T bp = cell_beta<T, TC, KIND, OM1>(P, gxr, gy0c, lW, lS, om_p);
    const T bq = cell_beta<T, TC, KIND, OM1>(P, gxr, gyq, lW, lN, om_q);
    const T cp = cell_beta<T, TC, KIND, OM1>(P, gx0c, gyc, lW, lS, om_p);
    const T cr = cell_beta<T, TC, KIND, OM1>(P, gxt, gyc, lE, lS, om_r);
    if (i < er.nrow) {
      ec[0][0][lane] = fma(-vr[1], bq, bp) * vr[0];
      ec[0][1][lane] = vr[3];
      ec[0][2][lane] = vr[4];
      ec[0][3][lane] = fma(-vr[2], bp, bq) * vr[0];
      ec[0][4][lane] = vr[5];
      ec[0][5][lane] = vr[6];
    }
    if (i < er.ncol) {
      ec[1][0][lane] = fma(-vc[1], cr, cp) * vc[0];
      ec[1][1][lane] = vc[3];
      ec[1][2][lane] = vc[4];
      ec[1][3][lane] = fma(-vc[2], cp, cr) * vc[0];
      ec[1][4][lane] = vc[5];
      ec[1][5][lane] = vc[6];
    }
    __syncwarp();
    if (lane == 0) mb_arrive(&prefull[c % PRE]);
  }
}

// Edge warp 2 ("chain"): the corner, then lanes 0/1 advance the start row and
// the twin row, lanes 2/3 the start column and the twin column, one position
// per step (two FMAs), storing the start row and column and handing them to
// the band warps in groups of ECH positions.
template <class T, class TC, int KIND, bool OM1>
__device__ __forceinline__ void edge_chain(const StagedP<T, TC>& P, const Geo& g, const Region& rg,
                                           const EdgeRange& er, unsigned slab_g, int j, T (*ecoef)[2][6][32],
                                           mbar_t* prefull, mbar_t* preempty, T* ring0, mbar_t* full0,
                                           mbar_t* empty0, T* colval, mbar_t* colfull, T (*egrp)[16], int lane) {
  const int lW = g.cx ? 1 : 0, lE = lW ^ 1, lS = g.cy ? 3 : 2, lN = lS ^ 1;
  const int cidx = g.cx | (g.cy << 1);
  const T om_p = P.om[cidx], om_q = P.om[cidx ^ 2], om_r = P.om[cidx ^ 1], om_s = P.om[cidx ^ 3];
  T self = T(0);  // lane 0: start-row cell, 1: twin-row cell, 2: start-column cell, 3: twin-column cell
  if (er.corner) {
    T p = T(0), q = T(0), r = T(0);
    if (lane == 0) {
      T hh[4], gx4[4], gy4[4], xx[4];
      const int sp = (1 ^ g.cx) | ((1 ^ g.cy) << 1), sq = (1 ^ g.cx) | (g.cy << 1);
      const int sr = g.cx | ((1 ^ g.cy) << 1), ss = g.cx | (g.cy << 1);
      const int gxa = g.gxl(0), gxb = g.gxl(-1), gya = g.gyl(0), gyb = g.gyl(-1);
      cell_g<T, TC>(P.c, (int64_t)gya * P.nx + gxa, lW, lS, OM1, om_p, gx4[sp], gy4[sp]);
      cell_g<T, TC>(P.c, (int64_t)gyb * P.nx + gxa, lW, lN, OM1, om_q, gx4[sq], gy4[sq]);
      cell_g<T, TC>(P.c, (int64_t)gya * P.nx + gxb, lE, lS, OM1, om_r, gx4[sr], gy4[sr]);
      cell_g<T, TC>(P.c, (int64_t)gyb * P.nx + gxb, lE, lN, OM1, om_s, gx4[ss], gy4[ss]);
      hh[sp] = cell_beta<T, TC, KIND, OM1>(P, gxa, gya, lW, lS, om_p);
      hh[sq] = cell_beta<T, TC, KIND, OM1>(P, gxa, gyb, lW, lN, om_q);
      hh[sr] = cell_beta<T, TC, KIND, OM1>(P, gxb, gya, lE, lS, om_r);
      hh[ss] = cell_beta<T, TC, KIND, OM1>(P, gxb, gyb, lE, lN, om_s);
      corner_solve(hh, gx4, gy4, xx);
      p = xx[sp];
      q = xx[sq];
      r = xx[sr];
      P.xnew[(int64_t)gya * P.nx + gxa] = p;
    }
    p = __shfl_sync(FULL, p, 0);
    q = __shfl_sync(FULL, q, 0);
    r = __shfl_sync(FULL, r, 0);
    self = lane == 1 ? q : (lane == 3 ? r : p);
  } else if (er.ncol > 0 && j > 0) {
    // start-column state at the last row of the previous slab
    if (!wait_gmem(&P.cflags[slab_g - 1], 1u, P.st)) return;
    if (lane == 2) self = __ldcg(P.chain + 2 * (slab_g - 1));
    if (lane == 3) self = __ldcg(P.chain + 2 * (slab_g - 1) + 1);
  }
  constexpr int ECH = HandOff<T>::ECH, NB = HandOff<T>::NB;
  const int line = lane >> 1, which = lane & 1;
  // A group's start-row / start-column values collect in egrp; after the
  // group, lanes q < ECH store them (start-row position i at rptr + i rstep,
  // start-column position i at cptr + i cstep), so that no global store sits
  // between two positions of the recurrence.
  T* const rout = P.xnew + (int64_t)g.gyl(0) * P.nx + g.gxl(er.k0);
  T* const cout = P.xnew + (int64_t)g.gyl(er.l_lo) * P.nx + g.gxl(0);
  const int64_t rstep = g.cx ? -1 : 1, cstep = g.cy ? -(int64_t)P.nx : (int64_t)P.nx;
  const bool row_lane = lane == 0, col_lane = lane == 2;
  const bool row_ring = row_lane && er.row_consumer;
  for (int c = 0; c < er.nchunks; ++c) {
    if (!mb_wait(&prefull[c % PRE], (c / PRE) & 1, P.st)) return;
    T(*ec)[6][32] = ecoef[c % PRE];
    const int nrow = max(0, min(32, er.nrow - 32 * c)), ncol = max(0, min(32, er.ncol - 32 * c));
    const int n = max(nrow, ncol);
    const int nmine = line == 0 ? nrow : ncol;
    for (int g8 = 0; g8 * ECH < n; ++g8) {
      const int i0 = 32 * c + ECH * g8;  // first position of this group
      if (er.row_consumer && ECH * g8 < nrow && i0 >= RING) {  // ring slots of the group free again
        if (!mb_wait(&empty0[(i0 / ECH) % NB], ((i0 / RING) - 1) & 1, P.st)) return;
      }
      // the group's coefficients into registers first, so that only the
      // shuffle and two FMAs separate consecutive positions
      T Ar[ECH], Br[ECH], Cr[ECH], xv[ECH];
      const int lq = lane < 4 ? lane : 0;
#pragma unroll
      for (int q = 0; q < ECH; ++q) {
        Ar[q] = ec[lq >> 1][(lq & 1) * 3 + 0][ECH * g8 + q];
        Br[q] = ec[lq >> 1][(lq & 1) * 3 + 1][ECH * g8 + q];
        Cr[q] = ec[lq >> 1][(lq & 1) * 3 + 2][ECH * g8 + q];
      }
#pragma unroll
      for (int q = 0; q < ECH; ++q) {
        const T other = __shfl_xor_sync(FULL, self, 1);
        const T nv = fma(Cr[q], other, fma(Br[q], self, Ar[q]));
        if (ECH * g8 + q < nmine) self = nv;
        xv[q] = self;
      }
#pragma unroll
      for (int q = 0; q < ECH; ++q) {
        const bool act = lane < 4 && ECH * g8 + q < nmine;
        if (act && (row_lane || col_lane)) egrp[line][q] = xv[q];
        if (act && row_ring) ring0[(i0 + q) & (RING - 1)] = xv[q];
        if (act && col_lane) colval[i0 + q] = xv[q];
      }
      // hand the group over (each value's writer arrives, so its stores are released)
      if (row_ring && ECH * g8 < nrow) mb_arrive(&full0[(i0 / ECH) % NB]);
      if (col_lane && ECH * g8 < ncol) mb_arrive(&colfull[i0 / ECH]);
      __syncwarp();
      if (lane < ECH) {
        const int jj = ECH * g8 + lane;
        if (jj < nrow) rout[(int64_t)(i0 + lane) * rstep] = egrp[0][lane];
        if (jj < ncol) cout[(int64_t)(i0 + lane) * cstep] = egrp[1][lane];
      }
      __syncwarp();
    }
    __syncwarp();
    if (lane == 0) mb_arrive(&preempty[c % PRE]);
  }
  // hand the start-column state to the next slab of this subdomain
  if (er.ncol > 0 && rg.slab_r0 + SLAB < rg.rhi) {
    if (lane == 2) P.chain[2 * slab_g] = self;
    if (lane == 3) P.chain[2 * slab_g + 1] = self;
    __syncwarp();
    if (lane == 0) {
      __threadfence();
      st_release(&P.cflags[slab_g], 1u);
    }
  }
}

template <bool B>
struct BoolC {
  static constexpr bool value = B;
};

struct BandShared {
  void* ring;      // [NW][RING] values
  mbar_t* full;    // [NW][NB]
  mbar_t* empty;   // [NW][NB]
  void* colval;    // [SLAB]
  mbar_t* colfull; // [SLAB / ECH]
  unsigned char* dsm;
};

// One band warp of one slab (lane = row), sweeping towards band column
// W - 1; DX = +1 / -1: global x grows / shrinks with the band column.
template <int DX, class T, class TC, int KIND, bool OM1>
__device__ __forceinline__ void band_run(const StagedP<T, TC>& P, const Geo& g, const Region& rg, bool tx, bool ty,
                                         int j, unsigned slab_g, int warp, int lane, const BandShared& sh) {
  using C = Cfg<T, TC, KIND>;
  constexpr int CH = C::CH, NS = C::NS, PITCH = C::PITCH, RP = C::ROWS * C::PITCH;
  constexpr int CS = C::NC * RP, VS = C::NV * RP, RPI = 32 / CH;
  constexpr int ECH = HandOff<T>::ECH, NB = HandOff<T>::NB;
  const int row0 = rg.slab_r0 + warp * BH;
  const int nrows = min(BH, rg.rhi - row0);
  const int W = rg.W;
  if (nrows <= 0 || W <= 0) return;
  // south input of lane 0: 0 none, 1 shared ring filled by the band below or
  // the edge warps, 2 the previous slab's top row in global memory
  const int in_kind = warp > 0 ? 1 : (j > 0 ? 2 : (ty ? 1 : 0));
  const bool more_rows = row0 + BH < rg.rhi;
  const int out_kind = (more_rows && warp + 1 < NW) ? 1 : ((more_rows && warp == NW - 1) ? 2 : 0);
  const bool use_col = tx;  // column clo - 1 comes from the edge warps
  const T om = P.om[g.cx | (g.cy << 1)];
  T* ring_in = reinterpret_cast<T*>(sh.ring) + warp * RING;
  T* ring_out = reinterpret_cast<T*>(sh.ring) + ((warp + 1) % NW) * RING;
  mbar_t* full_in = sh.full + warp * NBMAX;
  mbar_t* empty_in = sh.empty + warp * NBMAX;
  mbar_t* full_out = sh.full + ((warp + 1) % NW) * NBMAX;
  mbar_t* empty_out = sh.empty + ((warp + 1) % NW) * NBMAX;
  const T* colval = reinterpret_cast<const T*>(sh.colval);
  TC* cbuf = reinterpret_cast<TC*>(sh.dsm + warp * C::WARP_BYTES);
  T* vbuf = reinterpret_cast<T*>(sh.dsm + warp * C::WARP_BYTES + C::COEF_BYTES);
  T* xo = reinterpret_cast<T*>(sh.dsm + warp * C::WARP_BYTES + C::COEF_BYTES + C::VEC_BYTES);

  const bool row_on = lane < nrows;
  const int ly = row0 + (row_on ? lane : 0);
  const T* const inrow = P.xnew + (int64_t)g.gyl(in_kind == 2 ? row0 - 1 : ly) * P.nx + g.gxl(rg.clo);
  const bool lane0_in = in_kind != 0 && lane == 0;
  const bool lane31_out = out_kind == 1 && lane == BH - 1;
  // SOR: north neighbour inside the grid; band columns with an east neighbour: c < e_last
  const bool n_in = (g.gyl(ly + 1) >= 0) && (g.gyl(ly + 1) < P.ny);
  const int e_last = ((g.cx ? g.gx0 > 0 : g.gx0 + g.w < P.nx) ? g.w : g.w - 1) - rg.clo;

  // Copy plan: lane l copies column jl = l % CH of rows r0 + RPI i of every
  // chunk (row r's chunk k covers band columns kCH - r .. kCH - r + CH - 1);
  // element i of chunk k has band column kCH + jl - r0 - RPI i and global
  // index gbase + k DX CH + i istep. The chunk's results go back the same
  // way (row segments of CH values), not one row per lane and step.
  const int jl = lane % CH, r0c = lane / CH, lx0 = jl - r0c;
  const int rows_left = nrows - r0c;
  const int nrows_c = rows_left <= 0 ? 0 : (rows_left + RPI - 1) / RPI;
  const int gbase = g.gyl(row0 + r0c) * P.nx + g.gxl(rg.clo) + DX * lx0;
  const int istep = (g.cy ? -1 : 1) * RPI * P.nx - DX * RPI;
  const int sdst = r0c * PITCH + jl;
  const TC* src[C::NC];
  {
    const int lW = g.cx ? 1 : 0, lS = g.cy ? 3 : 2;
    if (KIND == KIND_TRI_UNIT) {
      src[0] = P.c[lW];
      src[1] = P.c[lS];
    } else {
      src[0] = P.inv;
      src[1] = P.c[lW];
      src[2 % C::NC] = P.c[lS];
      if (KIND == KIND_SOR) {
        src[3 % C::NC] = P.c[lW ^ 1];
        src[4 % C::NC] = P.c[lS ^ 1];
      }
    }
  }
  auto issue = [&](int k) {
    const int stg = k % NS;
    TC* cb = cbuf + stg * CS + sdst;
    T* vb = vbuf + stg * VS + sdst;
    const int ck = k * CH + lx0;
    const int gk = gbase + k * (DX * CH);
#pragma unroll
    for (int i = 0; i < CH; ++i) {
      if (i < nrows_c && (unsigned)(ck - RPI * i) < (unsigned)W) {
        const int gi = gk + i * istep;
#pragma unroll
        for (int a = 0; a < C::NC; ++a) cp_async<sizeof(TC)>(cb + a * RP + RPI * i * PITCH, src[a] + gi);
        cp_async<sizeof(T)>(vb + RPI * i * PITCH, P.rhs + gi);
      }
    }
    if (KIND == KIND_SOR) {
      // old values: own rows plus the row above (north), and one column beyond (east)
      T* ob = vbuf + stg * VS + RP;
      for (int e = lane; e < (BH + 1) * (CH + 1); e += 32) {
        const int r = e / (CH + 1), jc = e - r * (CH + 1);
        const int lyy = row0 + r, lx = rg.clo + k * CH - r + jc;
        if (lx < 0 || lx > g.w || lyy > g.h) continue;
        const int gx = g.gxl(lx), gy = g.gyl(lyy);
        if (gx < 0 || gx >= P.nx || gy < 0 || gy >= P.ny) continue;
        cp_async<sizeof(T)>(ob + r * PITCH + jc, P.xold + (int64_t)gy * P.nx + gx);
      }
    }
  };

  const int steps = W + nrows - 1;
  const int nchunks = (steps + CH - 1) / CH;
#pragma unroll
  for (int cc = 0; cc < NS - 1; ++cc) {
    if (cc < nchunks) issue(cc);
    cp_async_commit();
  }
  T x_prev = T(0);  // west value (0 before the first column: boundary, or the given start column)
  for (int k = 0; k < nchunks; ++k) {
    const int s0 = k * CH;
    __syncwarp();
    if (k + NS - 1 < nchunks) issue(k + NS - 1);
    cp_async_commit();
    // ---- hand-offs for this chunk (steps s0 .. s0 + CH - 1)
    bool ok = true;
    if (in_kind == 1) {
#pragma unroll
      for (int q = 0; q < CH / ECH; ++q) {
        const int s = s0 + ECH * q;
        if (s < W) ok = ok && mb_wait(&full_in[(s / ECH) % NB], (s / RING) & 1, P.st);
      }
    } else if (in_kind == 2 && s0 < W) {
      ok = wait_gmem(&P.flags[slab_g - 1], (unsigned)min(s0 + CH, W), P.st);
      if (ok && lane < CH && s0 + lane < W) ring_in[(s0 + lane) & (RING - 1)] = __ldcg(inrow + DX * (s0 + lane));
    }
    if (use_col && s0 < nrows) {  // start-column values of the lanes that begin in this chunk
#pragma unroll
      for (int q = 0; q < CH / ECH; ++q) {
        const int s = s0 + ECH * q;
        if (s < nrows) ok = ok && mb_wait(&sh.colfull[(warp * BH + s) / ECH], 0, P.st);
      }
      if (lane >= s0 && lane < s0 + CH && lane < nrows) x_prev = colval[warp * BH + lane];
    }
    if (out_kind == 1) {  // ring slots of the groups lane 31 starts in this chunk
#pragma unroll
      for (int q = 0; q < CH / ECH; ++q) {
        const int c = s0 - (BH - ECH) + ECH * q;
        if (c >= RING && c < W) ok = ok && mb_wait(&empty_out[(c / ECH) % NB], ((c / RING) - 1) & 1, P.st);
      }
    }
    cp_async_wait<NS - 1>();
    __syncwarp();
    if (!ok) {
      cp_async_wait<0>();
      return;
    }
    // ---- this chunk's operands into registers: x = beta - gW * xW - gS * xS
    T gWr[CH], gSr[CH], br[CH];
    {
      const TC* cb = cbuf + (k % NS) * CS + lane * PITCH;
      const T* vb = vbuf + (k % NS) * VS + lane * PITCH;
      const int ck = s0 - lane;  // this lane's band column at jj = 0
      constexpr int AS = RP;     // array stride in the stage
#pragma unroll
      for (int jj = 0; jj < CH; ++jj) {
        const TC* cj = cb + jj;
        if (KIND == KIND_TRI_SCALED) {
          const T inv = (T)cj[0];
          gWr[jj] = (T)cj[AS];
          gSr[jj] = (T)cj[2 * AS];
          br[jj] = OM1 ? inv * vb[jj] : P.bscale * inv * vb[jj];
        } else if (KIND == KIND_TRI_UNIT) {
          gWr[jj] = (T)cj[0];
          gSr[jj] = (T)cj[AS];
          br[jj] = vb[jj];
        } else {
          const T inv = (T)cj[0];
          gWr[jj] = (T)cj[AS];
          gSr[jj] = (T)cj[2 * AS];
          const T cE = (T)cj[3 * AS], cN = (T)cj[4 * AS];
          const T* ub = vb + RP;  // old values
          T acc = inv * vb[jj];
          if (ck + jj < e_last) acc = fma(-cE, ub[jj + 1], acc);
          if (n_in) acc = fma(-cN, ub[PITCH + jj + 1], acc);
          br[jj] = OM1 ? acc : fma(om, acc, (T(1) - om) * ub[jj]);
        }
        if (!OM1) {
          gWr[jj] *= om;
          gSr[jj] *= om;
        }
      }
    }
    T* const xo_l = xo + lane * PITCH;  // this lane's results of the chunk
    auto run = [&](auto ramp_tag) {
      constexpr bool RAMP = decltype(ramp_tag)::value;
#pragma unroll
      for (int jj = 0; jj < CH; ++jj) {
        const int s = s0 + jj;
        T r0 = T(0);
        if (lane0_in) r0 = ring_in[s & (RING - 1)];
        const T xs_sh = __shfl_up_sync(FULL, x_prev, 1);
        const T xS = lane == 0 ? r0 : xs_sh;
        const T x = fma(-gSr[jj], xS, fma(-gWr[jj], x_prev, br[jj]));
        const bool act = RAMP ? (row_on && (unsigned)(s - lane) < (unsigned)W) : row_on;
        xo_l[jj] = x;
        if (RAMP) {
          if (act) x_prev = x;
        } else {
          x_prev = x;
        }
        if (lane31_out && act) ring_out[(s - (BH - 1)) & (RING - 1)] = x;
      }
    };
    if (s0 >= nrows && s0 + CH <= W)
      run(BoolC<false>());
    else
      run(BoolC<true>());
    __syncwarp();
    {  // results of the chunk to global memory, row segments as in the copy plan
      const T* xr = xo + sdst;
      const int ck = s0 + lx0;
      const int gk = gbase + k * (DX * CH);
#pragma unroll
      for (int i = 0; i < CH; ++i)
        if (i < nrows_c && (unsigned)(ck - RPI * i) < (unsigned)W) P.xnew[gk + i * istep] = xr[RPI * i * PITCH];
    }
    // ---- hand-offs after this chunk: lane 31 finished band columns up to s0 + CH - BH
    if (out_kind == 1) {
      if (lane == BH - 1) {
#pragma unroll
        for (int q = 0; q < CH / ECH; ++q) {
          const int e = s0 - (BH - ECH) - 1 + ECH * q;  // last column of a group
          if (e >= 0 && e < W) mb_arrive(&full_out[(e / ECH) % NB]);
        }
        const int last = W - 1;  // a final partial group
        if (last % ECH != ECH - 1 && last >= s0 - (BH - 1) && last <= s0 + CH - BH)
          mb_arrive(&full_out[(last / ECH) % NB]);
      }
    } else if (out_kind == 2) {
      const int done = min(s0 + CH - (BH - 1), W);
      if (done > 0) {  // every lane stored part of the top row: fence each, then publish
        __threadfence();
        __syncwarp();
        if (lane == BH - 1) st_release(&P.flags[slab_g], (unsigned)done);
      }
    }
    if (in_kind == 1 && lane == 0) {  // lane 0 read the ring for steps s0 .. s0 + CH - 1
#pragma unroll
      for (int q = 0; q < CH / ECH; ++q) {
        const int s = s0 + ECH * q;
        if (s < W) mb_arrive(&empty_in[(s / ECH) % NB]);
      }
    }
  }
}

// One slab (CTA) of one sweep; `block` numbers the slabs of the sweep.
template <class T, class TC, int KIND, bool OM1>
__device__ __forceinline__ void staged_body(const StagedP<T, TC>& P, unsigned block) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ T inring[NW][RING];  // band w's south input: the row below its first row
  __shared__ T colval[SLAB];      // start-column values of the slab's band rows
  __shared__ T ecoef[PRE][2][6][32];
  __shared__ mbar_t full[NW][NBMAX], empty[NW][NBMAX], colfull[SLAB / 8], prefull[PRE], preempty[PRE];
  __shared__ T egrp[2][16];  // one group of start-row / start-column values
  __shared__ unsigned s_ticket;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int b = 0; b < NW; ++b)
      for (int q = 0; q < NBMAX; ++q) {
        mb_init(&full[b][q], 1);
        mb_init(&empty[b][q], 1);
      }
    for (int q = 0; q < SLAB / 8; ++q) mb_init(&colfull[q], 1);
    for (int q = 0; q < PRE; ++q) {
      mb_init(&prefull[q], 1);
      mb_init(&preempty[q], 1);
    }
    if (P.use_ticket) s_ticket = atomicAdd(P.ticket, 1u);
  }
  __syncthreads();
  const unsigned slab_id = P.use_ticket ? s_ticket : block;
  const unsigned sub = slab_id / P.spp;
  const int j = (int)(slab_id % P.spp);
  const int ix = (int)(sub % (unsigned)P.sx.p), iy = (int)(sub / (unsigned)P.sx.p);
  if (iy >= P.sy.p) return;
  bool tx, ty;
  const Geo g = subdomain_geo(P, ix, iy, tx, ty);
  const bool skip_x = P.rev && (g.cx ? (g.gx0 > 0) : (g.gx0 + g.w < P.nx));
  const bool skip_y = P.rev && (g.cy ? (g.gy0 > 0) : (g.gy0 + g.h < P.ny));
  Region rg;
  rg.rlo = ty ? 1 : 0;
  rg.rhi = g.h - (skip_y ? 1 : 0);
  rg.clo = tx ? 1 : 0;
  rg.chi = g.w - (skip_x ? 1 : 0);
  rg.W = rg.chi - rg.clo;
  rg.slab_r0 = rg.rlo + j * SLAB;
  rg.slab_rows = max(0, min(SLAB, rg.rhi - rg.slab_r0));
  if (j > 0 && rg.slab_rows == 0) return;
  const unsigned slab_g = sub * P.spp + j;

  if (warp >= NW) {
    if (tx || ty) {
      const EdgeRange er = edge_range(rg, tx, ty, j);
      if (warp == NW)
        edge_pre<T, TC, KIND, OM1>(P, g, ix, iy, er, ecoef, prefull, preempty, lane);
      else
        edge_chain<T, TC, KIND, OM1>(P, g, rg, er, slab_g, j, ecoef, prefull, preempty, inring[0], full[0],
                                     empty[0], colval, colfull, egrp, lane);
    }
    return;
  }
  BandShared sh;
  sh.ring = &inring[0][0];
  sh.full = &full[0][0];
  sh.empty = &empty[0][0];
  sh.colval = colval;
  sh.colfull = colfull;
  sh.dsm = dsm;
  if (g.cx)
    band_run<-1, T, TC, KIND, OM1>(P, g, rg, tx, ty, j, slab_g, warp, lane, sh);
  else
    band_run<1, T, TC, KIND, OM1>(P, g, rg, tx, ty, j, slab_g, warp, lane, sh);
}

template <class T, class TC, int KIND, bool OM1>
__global__ void __launch_bounds__((NW + 2) * 32, 2) sweep2d_staged_kernel(StagedP<T, TC> P) {
  staged_body<T, TC, KIND, OM1>(P, blockIdx.x);
}

// Several independent sweeps (one per problem of a batch) in one launch:
// problem p owns blocks off[p] .. off[p+1] - 1.
template <class T, class TC, int KIND, bool OM1>
__global__ void __launch_bounds__((NW + 2) * 32, 2)
    sweep2d_staged_batch_kernel(const StagedP<T, TC>* __restrict__ Pa, const unsigned* __restrict__ off, int np) {
  int lo = 0, hi = np - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= blockIdx.x) lo = mid;
    else hi = mid - 1;
  }
  staged_body<T, TC, KIND, OM1>(Pa[lo], blockIdx.x - off[lo]);
}

// Line table of one phase: one thread per start-row position (iy, gx) and per
// start-column position (ix, gy). The pair coefficients of Eq. 2d:sor2b2 in
// the recurrence form x_a(k) = A_a + B_a x_a(k-1) + C_a x_b(k-1):
//   det = 1 - g_ab g_ba, B_a = -g_a,prev / det, C_a = g_ab g_b,prev / det,
// and A_a = (beta_a - g_ab beta_b) / det evaluated in the sweep.
template <class T, class TC>
__global__ void line_table_kernel(StagedP<T, TC> P, T* tab, int om1) {
  const int64_t nrow = (int64_t)P.sy.p * P.nx, ncol = (int64_t)P.sx.p * P.ny;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nrow + ncol;
       e += (int64_t)gridDim.x * blockDim.x) {
    const bool is_row = e < nrow;
    int ix, iy, pos;
    if (is_row) {
      iy = (int)(e / P.nx);
      pos = (int)(e % P.nx);
      ix = split_find(P.sx, pos);
    } else {
      const int64_t f = e - nrow;
      ix = (int)(f / P.ny);
      pos = (int)(f % P.ny);
      iy = split_find(P.sy, pos);
    }
    bool tx, ty;
    const Geo g = subdomain_geo(P, ix, iy, tx, ty);
    const int lW = g.cx ? 1 : 0, lE = lW ^ 1, lS = g.cy ? 3 : 2, lN = lS ^ 1;
    const int cidx = g.cx | (g.cy << 1);
    T v[NT];
#pragma unroll
    for (int f = 0; f < NT; ++f) v[f] = T(0);
    if (is_row && ty) {
      const int gx = pos;
      T gpW, gpS, gqW, gqN;
      cell_g<T, TC>(P.c, (int64_t)g.gyl(0) * P.nx + gx, lW, lS, om1 != 0, P.om[cidx], gpW, gpS);
      cell_g<T, TC>(P.c, (int64_t)g.gyl(-1) * P.nx + gx, lW, lN, om1 != 0, P.om[cidx ^ 2], gqW, gqN);
      const T inv = rcp_rn(fma(-gpS, gqN, T(1)));
      v[0] = inv;
      v[1] = gpS;
      v[2] = gqN;
      v[3] = -gpW * inv;
      v[4] = (gpS * gqW) * inv;
      v[5] = -gqW * inv;
      v[6] = (gqN * gpW) * inv;
    } else if (!is_row && tx) {
      const int gy = pos;
      T gpW, gpS, grE, grS;
      cell_g<T, TC>(P.c, (int64_t)gy * P.nx + g.gxl(0), lW, lS, om1 != 0, P.om[cidx], gpW, gpS);
      cell_g<T, TC>(P.c, (int64_t)gy * P.nx + g.gxl(-1), lE, lS, om1 != 0, P.om[cidx ^ 1], grE, grS);
      const T inv = rcp_rn(fma(-gpW, grE, T(1)));
      v[0] = inv;
      v[1] = gpW;
      v[2] = grE;
      v[3] = -gpS * inv;
      v[4] = (gpW * grS) * inv;
      v[5] = -grS * inv;
      v[6] = (grE * gpS) * inv;
    }
    T* out = is_row ? tab + e : tab + NT * nrow + (e - nrow);
    const int64_t stride = is_row ? nrow : ncol;
#pragma unroll
    for (int f = 0; f < NT; ++f) out[f * stride] = v[f];
  }
}

template <class T, class TC, int KIND>
double staged_bytes(int64_t N) {
  int coefs = 0, vecs = 0;
  if (KIND == KIND_SOR) { coefs = 5; vecs = 3; }
  else if (KIND == KIND_TRI_SCALED) { coefs = 3; vecs = 2; }
  else { coefs = 2; vecs = 2; }
  return (double)N * (coefs * (double)sizeof(TC) + vecs * (double)sizeof(T));
}

template <class T, class TC, int KIND, bool OM1>
ndiag_status launch(Handle* h, const StagedP<T, TC>& P, unsigned nslabs) {
  using C = Cfg<T, TC, KIND>;
  static bool attr_set = false;
  if (!attr_set) {
    ND_CUDA(cudaFuncSetAttribute(sweep2d_staged_kernel<T, TC, KIND, OM1>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::BYTES));
    attr_set = true;
  }
  if (P.use_ticket) ND_CUDA(cudaMemsetAsync(h->sync, 0, h->sync_bytes, h->stream));
  const int slot = prof_begin(h);
  ++h->launches;
  ++h->sweep_launches;
  sweep2d_staged_kernel<T, TC, KIND, OM1><<<nslabs, (NW + 2) * 32, C::BYTES, h->stream>>>(P);
  ND_CUDA(cudaGetLastError());
  prof_end(h, slot, staged_bytes<T, TC, KIND>((int64_t)P.nx * P.ny));
  return NDIAG_OK;
}

// The line table of (set, phase, relaxation), built on first use and rebuilt
// when the set's values change.
template <class T, class TC>
ndiag_status line_table(Handle* h, const ScaledSet& set, StagedP<T, TC>& P, bool om1, const double* om) {
  LineTable* tab = nullptr;
  for (LineTable& t : h->line_tables) {
    if (t.set_base != set.base || t.base != P.base || t.om1 != (int)om1) continue;
    bool same = true;
    for (int k = 0; k < 4 && !om1; ++k) same = same && t.om[k] == om[k];
    if (same) {
      tab = &t;
      break;
    }
  }
  const int64_t nrow = (int64_t)P.sy.p * P.nx, ncol = (int64_t)P.sx.p * P.ny;
  const size_t bytes = sizeof(T) * NT * (size_t)(nrow + ncol);
  bool build = false;
  if (!tab) {
    LineTable t;
    t.set_base = set.base;
    t.base = P.base;
    t.om1 = om1 ? 1 : 0;
    for (int k = 0; k < 4; ++k) t.om[k] = om1 ? 1.0 : om[k];
    t.buf = dev_alloc(bytes, h->stream);
    if (!t.buf) return NDIAG_ENOMEM;
    t.bytes = bytes;
    h->line_tables.push_back(t);
    tab = &h->line_tables.back();
    build = true;
  }
  if (build || tab->set_version != set.version) {
    tab->set_version = set.version;
    const int64_t n = nrow + ncol;
    const int grid = (int)std::min<int64_t>((n + 255) / 256, (int64_t)h->sm_count * 8);
    ++h->launches;
    line_table_kernel<T, TC><<<grid, 256, 0, h->stream>>>(P, (T*)tab->buf, om1 ? 1 : 0);
    ND_CUDA(cudaGetLastError());
  }
  P.rowtab = (const T*)tab->buf;
  P.coltab = P.rowtab + NT * nrow;
  P.rt_stride = nrow;
  P.ct_stride = ncol;
  return NDIAG_OK;
}

template <class T, class TC>
ndiag_status make_params(Handle* h, int mode, int64_t t, const double* omega, const ScaledSet& set,
                         const void* rhs, const void* xold, void* xnew, double beta_scale, bool rev,
                         StagedP<T, TC>& P, unsigned& nslabs, bool& om1_out) {
  P = StagedP<T, TC>{};
  P.nx = (int)h->n[0];
  P.ny = (int)h->n[1];
  const bool nat = mode == NDIAG_NATURAL || mode == MODE_NATURAL_REV;
  const int px = nat ? 1 : h->sub[0], py = nat ? 1 : h->sub[1];
  P.sx = Split{px, P.nx / px, P.nx % px};
  P.sy = Split{py, P.ny / py, P.ny % py};
  P.base = nat ? (mode == MODE_NATURAL_REV ? 3 : 0) : base_corner(2, t);
  P.coupled = (nat || rev) ? 0 : 1;
  P.rev = rev ? 1 : 0;
  const int bands = (P.sy.len(0) + BH - 1) / BH;
  P.spp = (bands + NW - 1) / NW;
  P.use_ticket = P.spp > 1;
  const size_t N = (size_t)h->N;
  const TC* base = (const TC*)set.base;
  P.inv = base;
  for (int e = 0; e < 4; ++e) P.c[e] = base + (size_t)(1 + e) * N;
  P.rhs = (const T*)rhs;
  P.xold = (const T*)xold;
  P.xnew = (T*)xnew;
  bool om1 = true;
  double om_used[4];
  for (int k = 0; k < 4; ++k) {
    const double w = omega ? (nat ? omega[0] : omega[k]) : 1.0;
    om_used[k] = w;
    P.om[k] = (T)w;
    if (w != 1.0) om1 = false;
  }
  const bool om1_g = om1;  // the line table depends on the couplings' scaling only
  P.bscale = (T)beta_scale;
  if (beta_scale != 1.0) om1 = false;
  if (P.coupled) ND_TRY(line_table(h, set, P, om1_g, om_used));
  nslabs = (unsigned)(px * py * P.spp);
  if (P.use_ticket) {
    const size_t need = sizeof(unsigned) * (1 + 2 * (size_t)nslabs);
    const size_t need_ch = sizeof(T) * 2 * (size_t)nslabs;
    if (need > h->sync_bytes) {
      if (h->sync) dev_free(h->sync, h->sync_bytes, h->stream);
      h->sync = (unsigned*)dev_alloc(need, h->stream);
      h->sync_bytes = h->sync ? need : 0;
      if (!h->sync) return NDIAG_ENOMEM;
    }
    if (need_ch > h->twin_hand_bytes) {
      if (h->twin_hand) dev_free(h->twin_hand, h->twin_hand_bytes, h->stream);
      h->twin_hand = dev_alloc(need_ch, h->stream);
      h->twin_hand_bytes = h->twin_hand ? need_ch : 0;
      if (!h->twin_hand) return NDIAG_ENOMEM;
    }
    P.ticket = h->sync;
    P.flags = h->sync + 1;
    P.cflags = h->sync + 1 + nslabs;
    P.chain = (T*)h->twin_hand;
  }
  P.st = h->status;
  om1_out = om1;
  return NDIAG_OK;
}

template <class T, class TC>
ndiag_status fill(Handle* h, int kind, int mode, int64_t t, const double* omega, const ScaledSet& set,
                  const void* rhs, const void* xold, void* xnew, double beta_scale, bool rev) {
  StagedP<T, TC> P;
  unsigned nslabs = 0;
  bool om1 = true;
  ND_TRY(make_params(h, mode, t, omega, set, rhs, xold, xnew, beta_scale, rev, P, nslabs, om1));
  if (kind == KIND_SOR)
    return om1 ? launch<T, TC, KIND_SOR, true>(h, P, nslabs) : launch<T, TC, KIND_SOR, false>(h, P, nslabs);
  if (kind == KIND_TRI_SCALED)
    return om1 ? launch<T, TC, KIND_TRI_SCALED, true>(h, P, nslabs)
               : launch<T, TC, KIND_TRI_SCALED, false>(h, P, nslabs);
  if (kind == KIND_TRI_UNIT)
    return om1 ? launch<T, TC, KIND_TRI_UNIT, true>(h, P, nslabs)
               : launch<T, TC, KIND_TRI_UNIT, false>(h, P, nslabs);
  return NDIAG_EINVAL;
}


template <class T, class TC, int KIND, bool OM1>
ndiag_status launch_batch(const BatchSweep& b, cudaStream_t s) {
  using C = Cfg<T, TC, KIND>;
  static bool attr_set = false;
  if (!attr_set) {
    ND_CUDA(cudaFuncSetAttribute(sweep2d_staged_batch_kernel<T, TC, KIND, OM1>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::BYTES));
    attr_set = true;
  }
  sweep2d_staged_batch_kernel<T, TC, KIND, OM1><<<b.total, (NW + 2) * 32, C::BYTES, s>>>(
      (const StagedP<T, TC>*)b.params, b.off, b.np);
  ND_CUDA(cudaGetLastError());
  return NDIAG_OK;
}

template <class T, class TC>
ndiag_status batch_prepare_t(BatchSweep& b, Handle* const* hs, int np, int kind, int mode, int64_t t,
                             const double* omega, int set_sel, const void* const* rhs, const void* const* xold,
                             void* const* xnew, double beta_scale, bool rev, cudaStream_t s) {
  std::vector<StagedP<T, TC>> ps((size_t)np);
  std::vector<unsigned> off((size_t)np + 1, 0);
  bool om1_all = true;
  for (int p = 0; p < np; ++p) {
    Handle* h = hs[p];
    const ScaledSet& set = set_sel == 0 ? h->sor : (set_sel == 1 ? h->ilu : h->sorT);
    unsigned ns = 0;
    bool om1 = true;
    ND_TRY(make_params(h, mode, t, omega, set, rhs[p], xold ? xold[p] : nullptr, xnew[p], beta_scale, rev, ps[p],
                       ns, om1));
    if (ps[p].use_ticket) {
      set_error("batched sweeps need subdomains of at most 128 rows");
      return NDIAG_EINVAL;
    }
    if (p == 0) om1_all = om1;
    if (om1 != om1_all) return NDIAG_EINVAL;
    off[p + 1] = off[p] + ns;
  }
  const size_t pb = sizeof(StagedP<T, TC>) * (size_t)np, ob = sizeof(unsigned) * (size_t)(np + 1);
  if (pb > b.params_bytes) {
    dev_free(b.params, b.params_bytes, s);
    b.params = dev_alloc(pb, s);
    b.params_bytes = b.params ? pb : 0;
  }
  if (ob > b.off_bytes) {
    dev_free(b.off, b.off_bytes, s);
    b.off = (unsigned*)dev_alloc(ob, s);
    b.off_bytes = b.off ? ob : 0;
  }
  if (!b.params || !b.off) return NDIAG_ENOMEM;
  b.host_params.resize(pb);
  std::memcpy(b.host_params.data(), ps.data(), pb);
  b.host_off = off;
  ND_CUDA(cudaMemcpyAsync(b.params, b.host_params.data(), pb, cudaMemcpyHostToDevice, s));
  ND_CUDA(cudaMemcpyAsync(b.off, b.host_off.data(), ob, cudaMemcpyHostToDevice, s));
  b.np = np;
  b.total = off[np];
  b.kind = kind;
  b.om1 = om1_all;
  b.precision = hs[0]->precision;
  double bytes = 0.0;
  for (int p = 0; p < np; ++p) {
    const int64_t N = hs[p]->N;
    bytes += kind == KIND_SOR ? staged_bytes<T, TC, KIND_SOR>(N)
                              : (kind == KIND_TRI_SCALED ? staged_bytes<T, TC, KIND_TRI_SCALED>(N)
                                                         : staged_bytes<T, TC, KIND_TRI_UNIT>(N));
  }
  b.bytes = bytes;
  return NDIAG_OK;
}

template <class T, class TC>
ndiag_status batch_launch_t(const BatchSweep& b, cudaStream_t s) {
  if (b.kind == KIND_SOR) return b.om1 ? launch_batch<T, TC, KIND_SOR, true>(b, s) : launch_batch<T, TC, KIND_SOR, false>(b, s);
  if (b.kind == KIND_TRI_SCALED)
    return b.om1 ? launch_batch<T, TC, KIND_TRI_SCALED, true>(b, s) : launch_batch<T, TC, KIND_TRI_SCALED, false>(b, s);
  return b.om1 ? launch_batch<T, TC, KIND_TRI_UNIT, true>(b, s) : launch_batch<T, TC, KIND_TRI_UNIT, false>(b, s);
}

}  // namespace

ndiag_status batch_sweep_prepare(BatchSweep& b, Handle* const* hs, int np, int kind, int mode, int64_t t,
                                 const double* omega, int set_sel, const void* const* rhs, const void* const* xold,
                                 void* const* xnew, double beta_scale, bool rev, cudaStream_t s) {
  if (np < 1) return NDIAG_EINVAL;
  for (int p = 0; p < np; ++p)
    if (hs[p]->dim != 2 || hs[p]->stencil != 5 || hs[p]->precision != hs[0]->precision) return NDIAG_EINVAL;
  switch (hs[0]->precision) {
    case NDIAG_FP64:
      return batch_prepare_t<double, double>(b, hs, np, kind, mode, t, omega, set_sel, rhs, xold, xnew, beta_scale,
                                             rev, s);
    case NDIAG_FP32:
      return batch_prepare_t<float, float>(b, hs, np, kind, mode, t, omega, set_sel, rhs, xold, xnew, beta_scale,
                                           rev, s);
  }
  return NDIAG_EINVAL;
}

ndiag_status batch_sweep_launch(const BatchSweep& b, cudaStream_t s) {
  if (b.total == 0) return NDIAG_OK;
  return b.precision == NDIAG_FP64 ? batch_launch_t<double, double>(b, s) : batch_launch_t<float, float>(b, s);
}

void batch_sweep_free(BatchSweep& b, cudaStream_t s) {
  dev_free(b.params, b.params_bytes, s);
  dev_free(b.off, b.off_bytes, s);
  b = BatchSweep{};
}

// Returns NDIAG_EINVAL when this kernel does not cover the request (the
// caller then uses the single-pass kernel).
ndiag_status launch_sweep2d_staged(Handle* h, int kind, int mode, int64_t t, const double* omega,
                                   const ScaledSet& set, const void* rhs, const void* xold, void* xnew,
                                   double beta_scale, bool rev) {
  if (kind != KIND_SOR && kind != KIND_TRI_SCALED && kind != KIND_TRI_UNIT) return NDIAG_EINVAL;
  if (h->N > (int64_t)INT32_MAX / 2) return NDIAG_EINVAL;  // 32-bit cell offsets in the copy plans
  switch (h->precision) {
    case NDIAG_FP64:
      return fill<double, double>(h, kind, mode, t, omega, set, rhs, xold, xnew, beta_scale, rev);
    case NDIAG_FP32:
      return fill<float, float>(h, kind, mode, t, omega, set, rhs, xold, xnew, beta_scale, rev);
  }
  return NDIAG_EINVAL;
}

}  // namespace nd
