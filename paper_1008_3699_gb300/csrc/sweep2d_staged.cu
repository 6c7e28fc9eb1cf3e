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
//   (Eq. 2d:sor4b4) -- depend only on each other and on old values, so an
//   extra "edge" warp computes them ahead of the sweep. Its 32 lanes first
//   evaluate, for 32 positions at once, the pair coefficients of the line
//   written as a linear recurrence x_a(k) = A + B x_a(k-1) + C x_b(k-1); then
//   four lanes advance the row pair and the column pair together, two fp64
//   FMAs per position. Values go to the bands through shared memory (and, for
//   slabs further down the same subdomain, through global memory behind a
//   release/acquire flag). The CTA on the other side of the interface
//   evaluates the same recurrence with the roles swapped and the same
//   operations, so both sides agree bit for bit without synchronising.
// * Each band warp (lane = row) walks the columns as a skewed wavefront:
//   lane l handles column s - l at step s. Its operands are staged into
//   shared memory by cp.async in chunks of CH steps, skewed per row (row l's
//   chunk k covers columns kCH - l .. kCH - l + CH - 1), so a chunk is used
//   during exactly CH steps and NS stages give a lead of (NS - 1) CH steps.
//   Shared rows have an odd pitch, so the 32 lanes' reads are conflict-free.
//   Each chunk is unrolled, so shared-memory offsets are compile-time.
//   The west value is the lane's own previous result and the south value
//   arrives by shuffle; the west term is applied first, so the shuffle
//   latency overlaps the first FMA, and with unit relaxation a cell costs two
//   or three fp64 instructions (GB300 retires one fp64 warp instruction per
//   64 cycles per sub-partition, whatever the number of active lanes).
// * Bands of a slab hand their top row to the next band through a shared
//   ring published every ECH columns; slabs of a taller subdomain (the natural
//   ordering is one subdomain) through global memory and progress flags, the
//   slabs taken in ticket order. Every wait is bounded (NDIAG_ETIMEOUT).
#include "sweep_common.cuh"

namespace nd {
namespace {

using namespace sweep;

constexpr int NW = 4;          // band warps per CTA
constexpr int BH = 32;         // rows per band
constexpr int SLAB = NW * BH;  // rows per CTA
constexpr int RING = 64;       // band hand-off ring (columns)
constexpr int ECH = 8;         // hand-off chunk (columns): band to band, edge to band
constexpr int ERING = 64;      // start-row ring (columns)

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
  unsigned* ticket;
  unsigned* flags;   // per slab: columns of the top row published
  unsigned* cflags;  // per slab: start-column recurrence state published
  T* chain;          // per slab: that state (2 values)
  DevStatus* st;
};

template <class T, class TC, int KIND>
struct Cfg {
  static constexpr int CH = sizeof(T) == 8 ? 8 : 16;   // steps per chunk
  static constexpr int NS = sizeof(T) == 8 ? 2 : 3;    // stages
  static constexpr int NC = KIND == KIND_SOR ? 5 : (KIND == KIND_TRI_SCALED ? 3 : 2);
  static constexpr int NV = KIND == KIND_SOR ? 2 : 1;  // rhs (+ u_old)
  static constexpr int ROWS = KIND == KIND_SOR ? BH + 1 : BH;
  static constexpr int PITCH = CH + 1;                 // odd: conflict-free
  static constexpr size_t COEF_BYTES = align16(sizeof(TC) * NS * NC * ROWS * PITCH);
  static constexpr size_t VEC_BYTES = align16(sizeof(T) * NS * NV * ROWS * PITCH);
  static constexpr size_t WARP_BYTES = COEF_BYTES + VEC_BYTES;
  static constexpr size_t BYTES = NW * WARP_BYTES;
};

// beta and the implicit couplings of one cell (direct global loads; edge warps).
// jx / jy: entries (0 W, 1 E, 2 S, 3 N) of the cell's implicit x / y
// neighbour; the opposite entries hold old values (SOR only). The x term is
// taken before the y term so that every CTA evaluating a cell does the same.
template <class T, class TC, int KIND, bool OM1>
__device__ __forceinline__ void cell_bg(const StagedP<T, TC>& P, int gx, int gy, int jx, int jy, T om,
                                        T& beta, T& gjx, T& gjy) {
  const int64_t gi = (int64_t)gy * P.nx + gx;
  gjx = ldco<T, TC>(P.c[jx] + gi);
  gjy = ldco<T, TC>(P.c[jy] + gi);
  if (!OM1) {
    gjx *= om;
    gjy *= om;
  }
  if (KIND == KIND_SOR) {
    T acc = ldco<T, TC>(P.inv + gi) * __ldg(P.rhs + gi);
    const int ox = jx ^ 1, oy = jy ^ 1;
    const int xo = gx + (ox == 1 ? 1 : -1);
    if (xo >= 0 && xo < P.nx) acc = fma(-ldco<T, TC>(P.c[ox] + gi), __ldg(P.xold + gi + (xo - gx)), acc);
    const int yo = gy + (oy == 3 ? 1 : -1);
    if (yo >= 0 && yo < P.ny)
      acc = fma(-ldco<T, TC>(P.c[oy] + gi), __ldg(P.xold + gi + (int64_t)(yo - gy) * P.nx), acc);
    beta = OM1 ? acc : fma(om, acc, (T(1) - om) * __ldg(P.xold + gi));
  } else if (KIND == KIND_TRI_SCALED) {
    beta = ldco<T, TC>(P.inv + gi) * __ldg(P.rhs + gi);
    if (!OM1) beta *= P.bscale;
  } else {
    beta = __ldg(P.rhs + gi);
  }
}

struct Geo {
  int gx0, w, gy0, h, cx, cy;
  __device__ int gxl(int lx) const { return cx ? gx0 + w - 1 - lx : gx0 + lx; }
  __device__ int gyl(int ly) const { return cy ? gy0 + h - 1 - ly : gy0 + ly; }
};

struct EdgeShared {
  int rowp, rowc, colp;  // start-row values ready / taken by band 0; start-column values ready
  int pre, used;         // coefficient chunks precomputed / consumed by the chain warp
};

// Positions handled by the edge warps of one slab.
struct EdgeRange {
  bool corner, do_row, do_col;
  int k0, row_end, l0, l_lo, col_end, nchunks;
};

__device__ __forceinline__ EdgeRange edge_range(const Geo& g, bool tx, bool ty, int j, int slab_rows) {
  EdgeRange e;
  e.corner = tx && ty && j == 0;
  e.do_row = ty && j == 0;
  e.do_col = tx;
  e.l_lo = j * SLAB;
  e.k0 = e.corner ? 1 : 0;
  e.l0 = e.corner ? 1 : e.l_lo;
  e.row_end = e.do_row ? g.w : e.k0;
  e.col_end = e.do_col ? e.l_lo + slab_rows : e.l0;
  const int n = max(e.row_end - e.k0, e.col_end - e.l0);
  e.nchunks = (max(n, 0) + 31) / 32;
  return e;
}

// Per-lane copy plan of one band's chunks. A chunk holds CH columns of each of
// the band's 32 rows (row r's chunk k covers local columns kCH - r ..
// kCH - r + CH - 1). Lane l always copies column jl = l % CH of rows
// r0 + RPI i (r0 = l / CH, RPI = 32 / CH, i = 0..CH-1), so for chunk k the
// element's local column is kCH + jl - r0 - RPI i and its global index is
// base + k kstep + i istep: one multiply-add per element.
struct CopyPlan {
  int lx0;    // jl - r0
  int nrows;  // i < nrows: row inside the subdomain
  int base, kstep, istep;
  int sdst;   // shared offset of (row r0, column jl)
};

template <int CH, int PITCH>
__device__ __forceinline__ CopyPlan copy_plan(const Geo& g, int nx, int band, int lane) {
  constexpr int RPI = 32 / CH;
  CopyPlan c;
  const int jl = lane % CH, r0 = lane / CH;
  c.lx0 = jl - r0;
  const int rows_left = g.h - band * BH - r0;  // rows r0 + RPI i with i < ceil(rows_left / RPI)
  c.nrows = rows_left <= 0 ? 0 : (rows_left + RPI - 1) / RPI;
  const int dx = g.cx ? -1 : 1, dy = g.cy ? -1 : 1;
  const int gy_first = g.gyl(band * BH + r0);
  c.base = gy_first * nx + g.gxl(0) + dx * c.lx0;
  c.kstep = dx * CH;
  c.istep = dy * RPI * nx - dx * RPI;
  c.sdst = r0 * PITCH + jl;
  return c;
}

// Issue the cp.async copies of chunk k of one band into stage buffers.
template <class T, class TC, int KIND>
__device__ __forceinline__ void issue_chunk(const StagedP<T, TC>& P, const Geo& g, const CopyPlan& cp,
                                            const TC* const* src, int band, int k, TC* cb, T* vb, int lane) {
  using C = Cfg<T, TC, KIND>;
  constexpr int CH = C::CH, RPI = 32 / CH;
  const int lxk = k * CH + cp.lx0;
  const int gk = cp.base + k * cp.kstep;
#pragma unroll
  for (int i = 0; i < CH; ++i) {
    const int lx = lxk - RPI * i;
    if (i < cp.nrows && (unsigned)lx < (unsigned)g.w) {
      const int gi = gk + i * cp.istep;
      const int d = cp.sdst + RPI * i * C::PITCH;
#pragma unroll
      for (int a = 0; a < C::NC; ++a) cp_async<sizeof(TC)>(cb + a * C::ROWS * C::PITCH + d, src[a] + gi);
      cp_async<sizeof(T)>(vb + d, P.rhs + gi);
    }
  }
  if (KIND == KIND_SOR) {
    // old values: own rows plus the row above (north), and one column beyond (east)
    for (int e = lane; e < (BH + 1) * (CH + 1); e += 32) {
      const int r = e / (CH + 1), j = e - r * (CH + 1);
      const int ly = band * BH + r, lx = k * CH - r + j;
      if (lx < 0 || lx > g.w || ly > g.h) continue;
      const int gx = g.gxl(lx), gy = g.gyl(ly);
      if (gx < 0 || gx >= P.nx || gy < 0 || gy >= P.ny) continue;
      cp_async<sizeof(T)>(vb + (C::ROWS + r) * C::PITCH + j, P.xold + (int64_t)gy * P.nx + gx);
    }
  }
}

// Inline fast path of the bounded waits.
__device__ __forceinline__ bool wait_ge(const volatile int* p, int v, DevStatus* st) {
  if (*p >= v) {
    __threadfence_block();
    return true;
  }
  return wait_smem(p, v, st);
}

// Edge warp 1 ("pre"): for 32 positions of each coupled start line at a time,
// all lanes evaluate the pair coefficients of the line recurrence into a
// two-slot ring in shared memory.
template <class T, class TC, int KIND, bool OM1>
__device__ void edge_pre(const StagedP<T, TC>& P, const Geo& g, const EdgeRange& er, volatile EdgeShared* es,
                         T (*ecoef)[2][6][32], int lane) {
  const int lW = g.cx ? 1 : 0, lE = lW ^ 1, lS = g.cy ? 3 : 2, lN = lS ^ 1;
  const int cidx = g.cx | (g.cy << 1);
  const T om_p = P.om[cidx], om_q = P.om[cidx ^ 2], om_r = P.om[cidx ^ 1];
  for (int c = 0; c < er.nchunks; ++c) {
    if (c >= 2 && !wait_smem(&es->used, c - 1, P.st)) return;  // slot c % 2 free again
    T(*ec)[6][32] = ecoef[c & 1];
    const int kk = er.k0 + 32 * c + lane, ll = er.l0 + 32 * c + lane;
    if (kk < er.row_end) {
      T bp, gpW, gpS, bq, gqW, gqN, A, B, C;
      cell_bg<T, TC, KIND, OM1>(P, g.gxl(kk), g.gyl(0), lW, lS, om_p, bp, gpW, gpS);
      cell_bg<T, TC, KIND, OM1>(P, g.gxl(kk), g.gyl(-1), lW, lN, om_q, bq, gqW, gqN);
      line_coefs(bp, bq, gpW, gqW, gpS, gqN, A, B, C);
      ec[0][0][lane] = A; ec[0][1][lane] = B; ec[0][2][lane] = C;
      line_coefs(bq, bp, gqW, gpW, gqN, gpS, A, B, C);
      ec[0][3][lane] = A; ec[0][4][lane] = B; ec[0][5][lane] = C;
    }
    if (ll < er.col_end) {
      T bp, gpW, gpS, br, grE, grS, A, B, C;
      cell_bg<T, TC, KIND, OM1>(P, g.gxl(0), g.gyl(ll), lW, lS, om_p, bp, gpW, gpS);
      cell_bg<T, TC, KIND, OM1>(P, g.gxl(-1), g.gyl(ll), lE, lS, om_r, br, grE, grS);
      line_coefs(bp, br, gpS, grS, gpW, grE, A, B, C);
      ec[1][0][lane] = A; ec[1][1][lane] = B; ec[1][2][lane] = C;
      line_coefs(br, bp, grS, gpS, grE, gpW, A, B, C);
      ec[1][3][lane] = A; ec[1][4][lane] = B; ec[1][5][lane] = C;
    }
    __syncwarp();
    if (lane == 0) {
      __threadfence_block();
      es->pre = c + 1;
    }
  }
}

// Edge warp 2 ("chain"): the corner, then lanes 0/1 advance the start row and
// the twin row, lanes 2/3 the start column and the twin column, one position
// per step (two fp64 FMAs), handing the values to the band warps.
template <class T, class TC, int KIND, bool OM1>
__device__ void edge_chain(const StagedP<T, TC>& P, const Geo& g, const EdgeRange& er, unsigned slab_g,
                           int j, int slab_rows, volatile EdgeShared* es, T* rowring, T* colval,
                           T (*ecoef)[2][6][32], int lane) {
  const int lW = g.cx ? 1 : 0, lE = lW ^ 1, lS = g.cy ? 3 : 2, lN = lS ^ 1;
  const int cidx = g.cx | (g.cy << 1);
  const T om_p = P.om[cidx], om_q = P.om[cidx ^ 2], om_r = P.om[cidx ^ 1], om_s = P.om[cidx ^ 3];
  T self = T(0);  // lane 0: start-row cell, 1: twin-row cell, 2: start-column cell, 3: twin-column cell
  if (er.corner) {
    T p = T(0), q = T(0), r = T(0);
    if (lane == 0) {
      T bp, gpW, gpS, bq, gqW, gqN, br, grE, grS, bs, gsE, gsN;
      cell_bg<T, TC, KIND, OM1>(P, g.gxl(0), g.gyl(0), lW, lS, om_p, bp, gpW, gpS);
      cell_bg<T, TC, KIND, OM1>(P, g.gxl(0), g.gyl(-1), lW, lN, om_q, bq, gqW, gqN);
      cell_bg<T, TC, KIND, OM1>(P, g.gxl(-1), g.gyl(0), lE, lS, om_r, br, grE, grS);
      cell_bg<T, TC, KIND, OM1>(P, g.gxl(-1), g.gyl(-1), lE, lN, om_s, bs, gsE, gsN);
      const int sp = (1 ^ g.cx) | ((1 ^ g.cy) << 1), sq = (1 ^ g.cx) | (g.cy << 1);
      const int sr = g.cx | ((1 ^ g.cy) << 1), ss = g.cx | (g.cy << 1);
      T hh[4], gx4[4], gy4[4], xx[4];
      hh[sp] = bp; gx4[sp] = gpW; gy4[sp] = gpS;
      hh[sq] = bq; gx4[sq] = gqW; gy4[sq] = gqN;
      hh[sr] = br; gx4[sr] = grE; gy4[sr] = grS;
      hh[ss] = bs; gx4[ss] = gsE; gy4[ss] = gsN;
      corner_solve(hh, gx4, gy4, xx);
      p = xx[sp];
      q = xx[sq];
      r = xx[sr];
      rowring[0] = p;
      colval[0] = p;
      __threadfence_block();
      es->rowp = 1;
      es->colp = 1;
    }
    p = __shfl_sync(FULL, p, 0);
    q = __shfl_sync(FULL, q, 0);
    r = __shfl_sync(FULL, r, 0);
    self = lane == 1 ? q : (lane == 3 ? r : p);
  } else if (er.do_col && j > 0) {
    // start-column state at the last row of the previous slab
    if (!wait_gmem(&P.cflags[slab_g - 1], 1u, P.st)) return;
    if (lane == 2) self = __ldcg(P.chain + 2 * (slab_g - 1));
    if (lane == 3) self = __ldcg(P.chain + 2 * (slab_g - 1) + 1);
  }
  const int line = lane >> 1, which = lane & 1;
  for (int c = 0; c < er.nchunks; ++c) {
    if (!wait_smem(&es->pre, c + 1, P.st)) return;
    T(*ec)[6][32] = ecoef[c & 1];
    const int k_row = er.k0 + 32 * c, l_col = er.l0 + 32 * c;
    const int nrow = max(0, min(32, er.row_end - k_row)), ncol = max(0, min(32, er.col_end - l_col));
    if (nrow > 0 && k_row + nrow > ERING) {  // the bands must have taken the ring slots back
      if (!wait_smem(&es->rowc, k_row + nrow - ERING, P.st)) return;
    }
    const int n = max(nrow, ncol);
    for (int jj = 0; jj < n; ++jj) {
      const bool act = lane < 4 && jj < (line == 0 ? nrow : ncol);
      T A = T(0), B = T(0), C = T(0);
      if (act) {
        A = ec[line][which * 3 + 0][jj];
        B = ec[line][which * 3 + 1][jj];
        C = ec[line][which * 3 + 2][jj];
      }
      const T other = __shfl_xor_sync(FULL, self, 1);
      if (act) self = fma(C, other, fma(B, self, A));
      if (act && lane == 0) rowring[(k_row + jj) % ERING] = self;
      if (act && lane == 2) colval[l_col + jj - er.l_lo] = self;
      if ((jj + 1) % ECH == 0 || jj + 1 == n) {
        __threadfence_block();
        if (lane == 0 && nrow > 0) es->rowp = k_row + min(jj + 1, nrow);
        if (lane == 2 && ncol > 0) es->colp = l_col + min(jj + 1, ncol) - er.l_lo;
      }
    }
    __syncwarp();
    if (lane == 0) es->used = c + 1;
  }
  // hand the start-column state to the next slab of this subdomain
  if (er.do_col && slab_rows == SLAB && (j + 1) * SLAB < g.h) {
    if (lane == 2) P.chain[2 * slab_g] = self;
    if (lane == 3) P.chain[2 * slab_g + 1] = self;
    __syncwarp();
    if (lane == 0) {
      __threadfence();
      st_release(&P.cflags[slab_g], 1u);
    }
  }
}

template <class T, class TC, int KIND, bool OM1>
__global__ void __launch_bounds__((NW + 2) * 32) sweep2d_staged_kernel(StagedP<T, TC> P) {
  using C = Cfg<T, TC, KIND>;
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ T ring[NW][RING];
  __shared__ int prod[NW];
  __shared__ int cons[NW];
  __shared__ T rowring[ERING];
  __shared__ T colval[SLAB];
  __shared__ T ecoef[2][2][6][32];
  __shared__ EdgeShared es_raw;
  __shared__ unsigned s_ticket;
  volatile EdgeShared* es = &es_raw;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x < NW) {
    prod[threadIdx.x] = 0;
    cons[threadIdx.x] = 0;
  }
  if (threadIdx.x == 0) {
    es->rowp = 0;
    es->rowc = 0;
    es->colp = 0;
    es->pre = 0;
    es->used = 0;
    if (P.use_ticket) s_ticket = atomicAdd(P.ticket, 1u);
  }
  __syncthreads();
  const unsigned slab_id = P.use_ticket ? s_ticket : blockIdx.x;
  const unsigned sub = slab_id / P.spp, j = slab_id % P.spp;
  const int ix = (int)(sub % (unsigned)P.sx.p), iy = (int)(sub / (unsigned)P.sx.p);
  if (iy >= P.sy.p) return;
  Geo g;
  g.gx0 = P.sx.lo(ix);
  g.w = P.sx.len(ix);
  g.gy0 = P.sy.lo(iy);
  g.h = P.sy.len(iy);
  const int cidx = P.base ^ (ix & 1) ^ ((iy & 1) << 1);
  g.cx = cidx & 1;
  g.cy = (cidx >> 1) & 1;
  const bool tx = P.coupled && (g.cx ? (g.gx0 + g.w < P.nx) : (g.gx0 > 0));
  const bool ty = P.coupled && (g.cy ? (g.gy0 + g.h < P.ny) : (g.gy0 > 0));
  const int bands = (g.h + BH - 1) / BH;
  if ((int)j * NW >= bands) return;
  const int slab_rows = min(SLAB, g.h - (int)j * SLAB);
  const unsigned slab_g = sub * P.spp + j;

  if (warp >= NW) {
    if (tx || ty) {
      const EdgeRange er = edge_range(g, tx, ty, (int)j, slab_rows);
      if (warp == NW) edge_pre<T, TC, KIND, OM1>(P, g, er, es, ecoef, lane);
      else edge_chain<T, TC, KIND, OM1>(P, g, er, slab_g, (int)j, slab_rows, es, rowring, colval, ecoef, lane);
    }
    return;
  }
  const int band = (int)j * NW + warp;
  if (band >= bands) return;
  const bool skip_x = P.rev && (g.cx ? (g.gx0 > 0) : (g.gx0 + g.w < P.nx));
  const bool skip_y = P.rev && (g.cy ? (g.gy0 > 0) : (g.gy0 + g.h < P.ny));
  const bool use_row = ty && band == 0;  // lane 0 takes the start row from the edge warps
  const bool use_col = tx;               // column 0 comes from the edge warps
  const T om = P.om[cidx];
  constexpr int CH = C::CH, NS = C::NS, PITCH = C::PITCH, RP = C::ROWS * C::PITCH;
  constexpr int CS = C::NC * RP, VS = C::NV * RP;  // stage strides

  TC* cbuf = reinterpret_cast<TC*>(dsm + warp * C::WARP_BYTES);
  T* vbuf = reinterpret_cast<T*>(dsm + warp * C::WARP_BYTES + C::COEF_BYTES);

  const int ly = band * BH + lane;
  const bool row_on = ly < g.h && !(skip_y && ly == g.h - 1);
  const int wlim = (skip_x ? g.w - 1 : g.w);  // columns this lane computes: [0, wlim)
  const int gy = g.gyl(row_on ? ly : 0);
  const bool has_cons = band + 1 < bands;
  const bool smem_prod = has_cons && warp < NW - 1;
  const bool smem_cons = band > 0 && warp > 0;
  const bool gmem_cons = band > 0 && warp == 0;
  const int dx = g.cx ? -1 : 1;
  T* xrow = P.xnew + (int64_t)gy * P.nx + g.gxl(0);  // column lx is at xrow[dx * lx]
  // SOR: east / north neighbour inside the grid (old values)
  const bool n_in = (g.gyl(ly + 1) >= 0) && (g.gyl(ly + 1) < P.ny);
  const int e_last = (g.cx ? g.gx0 > 0 : g.gx0 + g.w < P.nx) ? g.w : g.w - 1;  // lx with an east neighbour: lx < e_last

  const int steps = g.w + BH - 1;
  const int nchunks = (steps + CH - 1) / CH;
  const CopyPlan cpl = copy_plan<CH, PITCH>(g, P.nx, band, lane);
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
#pragma unroll
  for (int cc = 0; cc < NS - 1; ++cc) {
    if (cc < nchunks) issue_chunk<T, TC, KIND>(P, g, cpl, src, band, cc, cbuf + cc * CS, vbuf + cc * VS, lane);
    cp_async_commit();
  }
  const int64_t dxb = (int64_t)dx;
  const bool need_i0 = smem_cons || gmem_cons || use_row;
  T x_prev = T(0);   // west value (0 before column 0: physical boundary or given column)
  T in0 = T(0);      // lane k < ECH: lane 0's input for step s0 + k (band below's top row, or the start row)
  T cv = T(0);       // column-0 value of this lane's row (edge warps)
  for (int k = 0; k < nchunks; ++k) {
    __syncwarp();
    if (k + NS - 1 < nchunks) {
      const int st = (k + NS - 1) % NS;
      issue_chunk<T, TC, KIND>(P, g, cpl, src, band, k + NS - 1, cbuf + st * CS, vbuf + st * VS, lane);
    }
    cp_async_commit();
    cp_async_wait<NS - 1>();
    __syncwarp();
    // ---- this chunk's operands into registers: x = beta - gW * xW - gS * xS
    T gWr[CH], gSr[CH], br[CH];
    {
      const TC* cb = cbuf + (k % NS) * CS + lane * PITCH;
      const T* vb = vbuf + (k % NS) * VS + lane * PITCH;
      const int lxk = k * CH - lane;  // this lane's column at jj = 0
#pragma unroll
      for (int jj = 0; jj < CH; ++jj) {
        if (KIND == KIND_TRI_SCALED) {
          const T inv = (T)cb[jj];
          gWr[jj] = (T)cb[RP + jj];
          gSr[jj] = (T)cb[2 * RP + jj];
          br[jj] = OM1 ? inv * vb[jj] : P.bscale * inv * vb[jj];
        } else if (KIND == KIND_TRI_UNIT) {
          gWr[jj] = (T)cb[jj];
          gSr[jj] = (T)cb[RP + jj];
          br[jj] = vb[jj];
        } else {
          const T inv = (T)cb[jj];
          gWr[jj] = (T)cb[RP + jj];
          gSr[jj] = (T)cb[2 * RP + jj];
          const T cE = (T)cb[3 * RP + jj], cN = (T)cb[4 * RP + jj];
          const T* ub = vb + RP;  // old values
          T acc = inv * vb[jj];
          if (lxk + jj < e_last) acc = fma(-cE, ub[jj + 1], acc);
          if (n_in) acc = fma(-cN, ub[PITCH + jj + 1], acc);
          br[jj] = OM1 ? acc : fma(om, acc, (T(1) - om) * ub[jj]);
        }
        if (!OM1) {
          gWr[jj] *= om;
          gSr[jj] *= om;
        }
      }
    }
    T* xk = xrow + dxb * (k * CH - lane);  // column lx = kCH + jj - lane at xk[dx * jj]
#pragma unroll
    for (int jj = 0; jj < CH; ++jj) {
      const int s = k * CH + jj;
      if (jj % ECH == 0) {
        // ---- lane 0's inputs for the next ECH steps
        if ((smem_cons || gmem_cons) && s < g.w) {
          const int need = min(s + ECH, g.w);
          const bool ok = smem_cons ? wait_ge(&prod[warp - 1], need, P.st)
                                    : wait_gmem(&P.flags[slab_g - 1], (unsigned)need, P.st);
          if (!ok) return;
          if (lane < ECH && s + lane < g.w) {
            if (smem_cons) in0 = ring[warp - 1][(s + lane) % RING];
            else in0 = __ldcg(P.xnew + (int64_t)g.gyl(band * BH - 1) * P.nx + g.gxl(s + lane));
          }
          __syncwarp();
          if (smem_cons && lane == 0) ((volatile int*)cons)[warp - 1] = need;
        } else if (use_row && s < g.w) {
          const int need = min(s + ECH, g.w);
          if (!wait_ge(&es->rowp, need, P.st)) return;
          if (lane < ECH && s + lane < g.w) in0 = rowring[(s + lane) % ERING];
          __syncwarp();
          if (lane == 0) es->rowc = need;
        }
        if (use_col && s < BH && warp * BH + s < slab_rows) {
          if (!wait_ge(&es->colp, min(warp * BH + s + ECH, slab_rows), P.st)) return;
          if (lane >= s && lane < s + ECH && ly < g.h) cv = colval[warp * BH + lane];
        }
        // ---- producer back-pressure on the shared ring (lane 31 writes column s - 31 on)
        if (smem_prod) {
          const int lx31 = s - (BH - 1);
          if (lx31 + ECH > RING && lx31 >= 0 && lx31 < g.w) {
            if (!wait_ge(&cons[warp], lx31 + ECH - RING, P.st)) return;
          }
        }
      }
      const T i0 = need_i0 ? __shfl_sync(FULL, in0, jj % ECH) : T(0);
      const T xS_sh = __shfl_up_sync(FULL, x_prev, 1);
      const int lx = s - lane;
      const T xS = lane > 0 ? xS_sh : i0;  // i0 = 0 for band 0 without a coupled start row
      T x = fma(-gSr[jj], xS, fma(-gWr[jj], x_prev, br[jj]));
      if (use_col && lx == 0) x = cv;           // start column, from the edge warps
      if (use_row && lane == 0) x = i0;         // start row, from the edge warps
      if (row_on && (unsigned)lx < (unsigned)wlim) {
        xk[dxb * jj] = x;
        x_prev = x;
        if (lane == BH - 1 && smem_prod) ring[warp][lx % RING] = x;
      }
      if (has_cons && lane == BH - 1) {
        // lane 31 finished column lx31; publish at multiples of ECH (a fixed jj, since
        // k CH is a multiple of ECH) and at the last column
        const int lx31 = s - (BH - 1);
        if ((jj % ECH == (ECH - 2 + ECH) % ECH && lx31 >= 0 && lx31 < g.w) || lx31 == g.w - 1) {
          if (smem_prod) {
            __threadfence_block();
            ((volatile int*)prod)[warp] = lx31 + 1;
          } else {
            __threadfence();
            st_release(&P.flags[slab_g], (unsigned)(lx31 + 1));
          }
        }
      }
    }
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

template <class T, class TC>
ndiag_status fill(Handle* h, int kind, int mode, int64_t t, const double* omega, const ScaledSet& set,
                  const void* rhs, const void* xold, void* xnew, double beta_scale, bool rev) {
  StagedP<T, TC> P{};
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
  for (int k = 0; k < 4; ++k) {
    const double w = omega ? (nat ? omega[0] : omega[k]) : 1.0;
    P.om[k] = (T)w;
    if (w != 1.0) om1 = false;
  }
  P.bscale = (T)beta_scale;
  if (beta_scale != 1.0) om1 = false;
  const unsigned nslabs = (unsigned)(px * py * P.spp);
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

}  // namespace

// Returns NDIAG_EINVAL when this kernel does not cover the request (the
// caller then uses the single-pass kernel).
ndiag_status launch_sweep2d_staged(Handle* h, int kind, int mode, int64_t t, const double* omega,
                                   const ScaledSet& set, const void* rhs, const void* xold, void* xnew,
                                   double beta_scale, bool rev) {
  if (kind != KIND_SOR && kind != KIND_TRI_SCALED && kind != KIND_TRI_UNIT) return NDIAG_EINVAL;
  switch (h->precision) {
    case NDIAG_FP64:
      return fill<double, double>(h, kind, mode, t, omega, set, rhs, xold, xnew, beta_scale, rev);
    case NDIAG_FP32:
      return fill<float, float>(h, kind, mode, t, omega, set, rhs, xold, xnew, beta_scale, rev);
  }
  return NDIAG_EINVAL;
}

}  // namespace nd
