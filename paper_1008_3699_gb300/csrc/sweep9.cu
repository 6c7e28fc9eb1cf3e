// Decomposed sequential sweep on 2D 9-point matrices (sm_103a), by levels.
//
// The paper calls the 9-point extension straightforward and gives no detail
// (Sec. 3). This library reads it as: inside a subdomain the cells are taken
// in lexicographic order of the reflected frame, so the new values of a cell
// are its W, SW, S and SE neighbours; across an interface only face
// neighbours couple, and only when both subdomains start at the interface
// (mutual, solved together as in Eqs. 2d:sor2b2 and 2d:sor4b4); diagonal
// neighbours across an interface keep their old values. With one subdomain
// this is natural-order SOR on the 9-point molecule.
//
// Level of own cell (x, y): x + 2y (SE = (x+1, y-1) then sits one level
// lower). One CTA per subdomain walks the levels; the block of a cell on a
// coupled start line holds its twins (2 or 4 cells, canonical order). An
// x-twin's SE neighbour is one column inside the neighbouring subdomain, so
// the two CTAs of an x-interface advance in step: before level L a CTA waits
// (bounded) until its x-neighbour has published level L - 1. All CTAs of the
// launch must be resident at once; the launcher checks that.
#include "sweep_common.cuh"

namespace nd {
namespace {

using namespace sweep;

constexpr int T9 = 256;

template <class T, class TC>
struct P9 {
  int nx, ny;
  Split sx, sy;
  int base, coupled;
  const TC* inv;
  const TC* c[8];  // scaled entries W E S N SW SE NW NE
  int64_t cn;      // c[e] == c[0] + e * cn: entries picked by arithmetic, not by indexing this block
  const T* rhs;
  const T* xold;
  T* xnew;
  T om[4];
  T bscale;
  unsigned* prog;  // per subdomain: levels completed (zeroed before the launch)
  DevStatus* st;
  // paired mode: the two subdomains of every coupled x-interface share one
  // CTA (half the threads each), so their lockstep is the CTA's own barrier
  int paired;
  int pair_par;    // parity of the x index that starts a pair
  int units;       // CTAs per row of subdomains
  int lmax_all;    // levels of the largest subdomain
  int half_elems;  // shared elements per subdomain (twin lines and ring)
};

// entry of the neighbour at local offset (dx, dy) for corner bits (cx, cy)
__device__ __forceinline__ int ent9(int dx, int dy, int cx, int cy) {
  const int gx = cx ? -dx : dx, gy = cy ? -dy : dy;
  if (gy == 0) return gx < 0 ? 0 : 1;
  if (gx == 0) return gy < 0 ? 2 : 3;
  if (gy < 0) return gx < 0 ? 4 : 5;
  return gx < 0 ? 6 : 7;
}

struct Sub9 {
  int ix, iy, g0[2], len[2], c[2], t[2];
  __device__ int gco(int a, int l) const { return c[a] ? g0[a] + len[a] - 1 - l : g0[a] + l; }
};

template <class T, class TC>
__device__ __forceinline__ Sub9 sub9(const P9<T, TC>& P, int ix, int iy) {
  Sub9 S;
  S.ix = ix;
  S.iy = iy;
  S.g0[0] = P.sx.lo(ix);
  S.len[0] = P.sx.len(ix);
  S.g0[1] = P.sy.lo(iy);
  S.len[1] = P.sy.len(iy);
  const int cidx = P.base ^ (ix & 1) ^ ((iy & 1) << 1);
  S.c[0] = cidx & 1;
  S.c[1] = (cidx >> 1) & 1;
  S.t[0] = P.coupled && (S.c[0] ? S.g0[0] + S.len[0] < P.nx : S.g0[0] > 0);
  S.t[1] = P.coupled && (S.c[1] ? S.g0[1] + S.len[1] < P.ny : S.g0[1] > 0);
  return S;
}

// Twin store: x-twins (-1, y) at [y], y-twins (x, -1) at [h + x], corner at [h + w].
__device__ __forceinline__ int slot9(int sub, const int* lc, int w, int h) {
  return sub == 1 ? lc[1] : (sub == 2 ? h + lc[0] : h + w);
}

// The block of own cell (x, y), which lies on the NC coupled start lines C:
// assembled member by member in canonical order, solved, the own member
// stored to xnew and the twins to the twin-line store.
// CM = the coupled lines as a compile-time mask (then C == CM), or 0: taken
// from C at run time; with the mask every axis index is a constant.
template <class T, class TC, int KIND, bool OM1, int NC, int CM = 0>
__device__ __forceinline__ T cell9(const P9<T, TC>& P, const Sub9& S, T* tw, int w, int h, int x, int y, int C) {
  const int own[2] = {x, y};
  int axes[2] = {0, 0}, nC = 0;
  if constexpr (CM != 0) {
    C = CM;
    axes[0] = (CM & 1) ? 0 : 1;
    axes[1] = 1;
    nC = NC;
  } else {
    for (int a = 0; a < 2; ++a)
      if (C >> a & 1) axes[nC++] = a;
  }
  constexpr int n = 1 << NC;  // nC == NC
  int mo = 0;
#pragma unroll
  for (int r = 0; r < NC; ++r)
    if (S.c[axes[r]] == 0) mo |= 1 << r;
  T M[n][n], hv[n];
  int64_t gidx[n];
#pragma unroll
  for (int m = 0; m < n; ++m) {
    int lc[2] = {own[0], own[1]}, sub = 0;
#pragma unroll
    for (int r = 0; r < NC; ++r)
      if (((m ^ mo) >> r) & 1) {
        lc[axes[r]] = -1;
        sub |= 1 << axes[r];
      }
    const int cm0 = S.c[0] ^ (sub & 1), cm1 = S.c[1] ^ ((sub >> 1) & 1);
    // extent of the member's subdomain and its local coordinates there
    int mlen[2], ml[2];
    for (int a = 0; a < 2; ++a) {
      if ((sub >> a) & 1) {
        const int ia = a == 0 ? (S.c[0] ? S.ix + 1 : S.ix - 1) : (S.c[1] ? S.iy + 1 : S.iy - 1);
        mlen[a] = a == 0 ? P.sx.len(ia) : P.sy.len(ia);
        ml[a] = 0;
      } else {
        mlen[a] = S.len[a];
        ml[a] = lc[a];
      }
    }
    const int gx = S.gco(0, lc[0]), gy = S.gco(1, lc[1]);
    const int64_t gi = (int64_t)gy * P.nx + gx;
    gidx[m] = gi;
    const T om = OM1 ? T(1) : P.om[cm0 | (cm1 << 1)];
#pragma unroll
    for (int k = 0; k < n; ++k) M[m][k] = T(0);
    M[m][m] = T(1);
    // explicit part (old values; SOR only) and the implicit part, each in
    // the member's own neighbour order, so every CTA forms the same terms
    T base = (KIND == KIND_TRI_UNIT) ? __ldg(P.rhs + gi) : ldco<T, TC>(P.inv + gi) * __ldg(P.rhs + gi);
    T impl = T(0);
    const int offs[8][2] = {{-1, 0}, {-1, -1}, {0, -1}, {1, -1}, {1, 0}, {1, 1}, {0, 1}, {-1, 1}};
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int dx = offs[q][0], dy = offs[q][1];
      const int qx = ml[0] + dx, qy = ml[1] + dy;
      const int e = ent9(dx, dy, cm0, cm1);
      const int ggx = gx + (cm0 ? -dx : dx), ggy = gy + (cm1 ? -dy : dy);
      if (ggx < 0 || ggx >= P.nx || ggy < 0 || ggy >= P.ny) continue;
      const bool upstream = q < 4;  // W, SW, S, SE
      const bool inside = qx >= 0 && qx < mlen[0] && qy >= 0 && qy < mlen[1];
      const int64_t gq = (int64_t)ggy * P.nx + ggx;
      if (upstream && inside) {
        // new value of a cell of the member's own subdomain
        T g = ldco<T, TC>(P.c[0] + e * P.cn + gi);
        if (!OM1) g *= om;
        T v;
        if (sub == 0) {
          v = __ldcg(P.xnew + gq);
        } else {
          // in S-coordinates: still on the twin line -> shared store, deeper -> global
          const int nl[2] = {lc[0] + (cm0 == S.c[0] ? dx : -dx), lc[1] + (cm1 == S.c[1] ? dy : -dy)};
          const bool on_line = ((sub & 1) ? nl[0] == -1 : nl[0] >= 0) && ((sub & 2) ? nl[1] == -1 : nl[1] >= 0);
          v = on_line ? tw[slot9(sub, nl, w, h)] : __ldcg(P.xnew + gq);
        }
        impl = fma(g, v, impl);
      } else if (upstream && (dx == 0 || dy == 0) && ((C >> (dx != 0 ? 0 : 1)) & 1)) {
        // face neighbour across a coupled start line: the block partner
        // partner index bit: the coupled axes in order (x before y)
        const int r = NC == 2 ? (dx != 0 ? 0 : 1) : 0;
        T g = ldco<T, TC>(P.c[0] + e * P.cn + gi);
        if (!OM1) g *= om;
        M[m][m ^ (1 << r)] = g;
      } else if (KIND == KIND_SOR) {
        // downstream neighbours, uncoupled or diagonal ones across an interface: old values
        base = fma(-ldco<T, TC>(P.c[0] + e * P.cn + gi), __ldg(P.xold + gq), base);
      }
    }
    T acc;
    if (KIND == KIND_SOR) acc = OM1 ? base : fma(om, base, (T(1) - om) * __ldg(P.xold + gi));
    else if (KIND == KIND_TRI_SCALED) acc = OM1 ? base : P.bscale * base;
    else acc = base;
    acc -= impl;
    hv[m] = acc;
  }
#pragma unroll
  for (int k = 0; k < n; ++k) {
    const T piv = M[k][k];
#pragma unroll
    for (int i = k + 1; i < n; ++i) {
      const T f = k == 0 ? M[i][k] : M[i][k] / piv;  // row 0 keeps its unit pivot
      if (f != T(0)) {
#pragma unroll
        for (int j = k + 1; j < n; ++j) M[i][j] = fma(-f, M[k][j], M[i][j]);
        hv[i] = fma(-f, hv[k], hv[i]);
      }
    }
  }
  T xs[n];
#pragma unroll
  for (int k = n - 1; k >= 0; --k) {
    T s = hv[k];
#pragma unroll
    for (int j = k + 1; j < n; ++j) s = fma(-M[k][j], xs[j], s);
    xs[k] = k == 0 ? s : s / M[k][k];
  }
#pragma unroll
  for (int m = 0; m < n; ++m) {
    if (m == mo) {
      P.xnew[gidx[m]] = xs[m];
    } else {
      int lc[2] = {own[0], own[1]}, sub = 0;
#pragma unroll
      for (int r = 0; r < NC; ++r)
        if (((m ^ mo) >> r) & 1) {
          lc[axes[r]] = -1;
          sub |= 1 << axes[r];
        }
      tw[slot9(sub, lc, w, h)] = xs[m];
    }
  }
  T own_x = xs[0];
#pragma unroll
  for (int m = 1; m < n; ++m)
    if (m == mo) own_x = xs[m];
  return own_x;
}

template <class T, class TC, int KIND, bool OM1>
__global__ void __launch_bounds__(T9) sweep9_kernel(P9<T, TC> P) {
  extern __shared__ __align__(16) unsigned char gsm[];
  T* tw = reinterpret_cast<T*>(gsm);
  int ix, iy, lt = threadIdx.x, stride = T9;
  bool active = true;
  if (P.paired) {  // unit k of row iy: subdomains start, start + 1 (or start alone)
    iy = (int)(blockIdx.x / (unsigned)P.units);
    const int k = (int)(blockIdx.x % (unsigned)P.units);
    const int start = P.pair_par == 0 ? 2 * k : (k == 0 ? 0 : 2 * k - 1);
    const int cnt = (P.pair_par == 1 && k == 0) ? 1 : min(2, P.sx.p - start);
    const int half = threadIdx.x >= T9 / 2 ? 1 : 0;
    active = half < cnt;
    ix = start + (active ? half : 0);
    lt = threadIdx.x - half * (T9 / 2);
    stride = T9 / 2;
    tw += half * P.half_elems;
  } else {
    ix = (int)(blockIdx.x % (unsigned)P.sx.p);
    iy = (int)(blockIdx.x / (unsigned)P.sx.p);
  }
  const Sub9 S = sub9(P, ix, iy);
  const int w = S.len[0], h = S.len[1];
  const int lmax = P.paired ? P.lmax_all : (w - 1) + 2 * (h - 1);
  const int tcode = S.t[0] | (S.t[1] << 1);
  // Pencil path (triangular kinds, h <= T9): thread y meets its row's next
  // cell x = L - 2y on every level. W is the row's previous cell (register);
  // SE, S, SW are row y - 1's cells of levels L - 1, L - 2, L - 3, kept in a
  // shared ring of four levels; the operands of the next level's one-cell
  // blocks are loaded before this level's arithmetic.
  const bool pen = KIND != KIND_SOR && h <= stride;
  T* ring = tw + (w + h + 1);  // [4][h]
  const int c0 = S.c[0], c1 = S.c[1];
  const int eW = ent9(-1, 0, c0, c1), eSW = ent9(-1, -1, c0, c1), eS = ent9(0, -1, c0, c1),
            eSE = ent9(1, -1, c0, c1);
  const TC *cW = P.c[0] + eW * P.cn, *cSW = P.c[0] + eSW * P.cn, *cS = P.c[0] + eS * P.cn,
           *cSE = P.c[0] + eSE * P.cn;
  const T om = OM1 ? T(1) : P.om[c0 | (c1 << 1)];
  const int y = lt;
  T ni = T(0), nr = T(0), ng[4] = {T(0), T(0), T(0), T(0)};  // next level's operands
  auto fetch = [&](int L2) {
    const int x2 = L2 - 2 * y;
    if (!pen || !active || y >= h || x2 < 0 || x2 >= w) return;
    if ((((x2 == 0) | ((y == 0) << 1)) & tcode) != 0) return;
    const int64_t gi = (int64_t)S.gco(1, y) * P.nx + S.gco(0, x2);
    if (KIND == KIND_TRI_SCALED) ni = ldco<T, TC>(P.inv + gi);
    nr = __ldg(P.rhs + gi);
    ng[0] = x2 >= 1 ? ldco<T, TC>(cW + gi) : T(0);
    ng[1] = (x2 >= 1 && y >= 1) ? ldco<T, TC>(cSW + gi) : T(0);
    ng[2] = y >= 1 ? ldco<T, TC>(cS + gi) : T(0);
    ng[3] = (x2 + 1 < w && y >= 1) ? ldco<T, TC>(cSE + gi) : T(0);
  };
  T xr = T(0);
  fetch(0);
  // x-neighbour across the coupled start line (its interior feeds the x-twins)
  const int nbx = S.c[0] ? ix + 1 : ix - 1;
  const unsigned* nprog = (S.t[0] && !P.paired) ? P.prog + (iy * P.sx.p + nbx) : nullptr;
  __shared__ int s_ok;
  if (threadIdx.x == 0) s_ok = 1;
  __syncthreads();
  for (int L = 0; L <= lmax; ++L) {
    if (nprog && L >= 2 && (L & 1) == 0 && L / 2 < h) {  // x-face block at this level
      if (threadIdx.x == 0 && s_ok) s_ok = wait_gmem(nprog, (unsigned)L, P.st) ? 1 : 0;
      __syncthreads();
      if (!s_ok) return;
    }
    if (pen) {
      const T ci = ni, cr = nr, cg0 = ng[0], cg1 = ng[1], cg2 = ng[2], cg3 = ng[3];
      if (L < lmax) fetch(L + 1);
      const int x = L - 2 * y;
      if (active && y < h && x >= 0 && x < w) {
        const int C = ((x == 0) | ((y == 0) << 1)) & tcode;
        T v;
        if (C == 0) {
          // the one-cell block, term for term as cell9: W, SW, S, SE
          T g[4] = {cg0, cg1, cg2, cg3};
          if (!OM1) {
#pragma unroll
            for (int q = 0; q < 4; ++q) g[q] *= om;
          }
          const T* rp = ring + (y - 1);
          T impl = T(0);
          if (x >= 1) impl = fma(g[0], xr, impl);
          if (x >= 1 && y >= 1) impl = fma(g[1], rp[((L - 3) & 3) * h], impl);
          if (y >= 1) impl = fma(g[2], rp[((L - 2) & 3) * h], impl);
          if (x + 1 < w && y >= 1) impl = fma(g[3], rp[((L - 1) & 3) * h], impl);
          T base = KIND == KIND_TRI_UNIT ? cr : ci * cr;
          T acc = (KIND == KIND_TRI_SCALED && !OM1) ? P.bscale * base : base;
          acc -= impl;
          P.xnew[(int64_t)S.gco(1, y) * P.nx + S.gco(0, x)] = acc;
          v = acc;
        } else if (C == 3) {
          v = cell9<T, TC, KIND, OM1, 2, 3>(P, S, tw, w, h, x, y, C);
        } else if (C == 1) {
          v = cell9<T, TC, KIND, OM1, 1, 1>(P, S, tw, w, h, x, y, C);
        } else {
          v = cell9<T, TC, KIND, OM1, 1, 2>(P, S, tw, w, h, x, y, C);
        }
        ring[(L & 3) * h + y] = v;
        xr = v;
      }
    } else {
      for (int y2 = lt; active && y2 < h; y2 += stride) {
        const int x = L - 2 * y2;
        if (x < 0 || x >= w) continue;
        const int C = ((x == 0) | ((y2 == 0) << 1)) & tcode;
        if (C == 0) cell9<T, TC, KIND, OM1, 0>(P, S, tw, w, h, x, y2, C);
        else if (C == 3) cell9<T, TC, KIND, OM1, 2>(P, S, tw, w, h, x, y2, C);
        else cell9<T, TC, KIND, OM1, 1>(P, S, tw, w, h, x, y2, C);
      }
    }
    __syncthreads();
    if (threadIdx.x == 0 && P.coupled && !P.paired) {
      __threadfence();
      st_release(P.prog + blockIdx.x, (unsigned)(L + 1));
    }
  }
}

// D-ILU pivots of the 9-point matrix: d_i = a_ii - sum over the implicit
// upstream cells j of the same subdomain (W, SW, S, SE) of a_ij a_ji / d_j.
__global__ void __launch_bounds__(T9) factor9_kernel(P9<double, double> P, const double* A, double* piv, int64_t N) {
  const int ix = (int)(blockIdx.x % (unsigned)P.sx.p), iy = (int)(blockIdx.x / (unsigned)P.sx.p);
  const Sub9 S = sub9(P, ix, iy);
  const int w = S.len[0], h = S.len[1];
  const int lmax = (w - 1) + 2 * (h - 1);
  const int offs[4][2] = {{-1, 0}, {-1, -1}, {0, -1}, {1, -1}};
  for (int L = 0; L <= lmax; ++L) {
    for (int y = threadIdx.x; y < h; y += T9) {
      const int x = L - 2 * y;
      if (x < 0 || x >= w) continue;
      const int gx = S.gco(0, x), gy = S.gco(1, y);
      const int64_t gi = (int64_t)gy * P.nx + gx;
      double di = A[gi];
      for (int q = 0; q < 4; ++q) {
        const int qx = x + offs[q][0], qy = y + offs[q][1];
        if (qx < 0 || qx >= w || qy < 0 || qy >= h) continue;
        const int e = ent9(offs[q][0], offs[q][1], S.c[0], S.c[1]);
        const int eb = ent9(-offs[q][0], -offs[q][1], S.c[0], S.c[1]);
        const int64_t gq = (int64_t)S.gco(1, qy) * P.nx + S.gco(0, qx);
        di -= A[(size_t)(1 + e) * N + gi] * A[(size_t)(1 + eb) * N + gq] / __ldcg(piv + gq);
      }
      if (di == 0.0) atomicExch(&P.st->zero_pivot, 1);
      piv[gi] = di;
    }
    __syncthreads();
  }
}

template <class T, class TC>
P9<T, TC> params9(Handle* h, int mode, int64_t t, const ScaledSet& set, const void* rhs, const void* xold,
                  void* xnew, unsigned& nsub) {
  P9<T, TC> P{};
  const bool nat = mode == NDIAG_NATURAL || mode == MODE_NATURAL_REV;
  P.nx = (int)h->n[0];
  P.ny = (int)h->n[1];
  const int px = nat ? 1 : h->sub[0], py = nat ? 1 : h->sub[1];
  P.sx = Split{px, P.nx / px, P.nx % px};
  P.sy = Split{py, P.ny / py, P.ny % py};
  P.base = nat ? (mode == MODE_NATURAL_REV ? 3 : 0) : base_corner(2, t);
  P.coupled = nat ? 0 : 1;
  const size_t N = (size_t)h->N;
  const TC* b = (const TC*)set.base;
  P.inv = b;
  for (int e = 0; e < 8; ++e) P.c[e] = b + (size_t)(1 + e) * N;
  P.cn = (int64_t)N;
  P.rhs = (const T*)rhs;
  P.xold = (const T*)xold;
  P.xnew = (T*)xnew;
  P.st = h->status;
  nsub = (unsigned)(px * py);
  return P;
}

template <class T, class TC, int KIND, bool OM1>
ndiag_status run9(Handle* h, P9<T, TC>& P, unsigned nsub, double bytes) {
  const int w = P.sx.len(0), hh = P.sy.len(0);
  // twin lines, then the pencil path's four-level ring (per subdomain)
  P.half_elems = w + hh + 1 + (hh <= T9 ? 4 * hh : 0);  // no ring where no row-per-thread pencil fits
  // pairing: coupled x-interfaces join ix and ix + 1 where ix has the parity
  // at which a subdomain starts at its max-x side
  P.paired = P.coupled && hh <= T9 / 2 && P.sx.p > 1;
  if (P.paired) {
    P.pair_par = (P.base & 1) ? 0 : 1;
    const int px = P.sx.p;
    P.units = P.pair_par == 0 ? (px + 1) / 2 : 1 + px / 2;
    P.lmax_all = (w - 1) + 2 * (hh - 1);
    nsub = (unsigned)(P.units * P.sy.p);
  }
  const size_t smem = sizeof(T) * (size_t)P.half_elems * (P.paired ? 2 : 1);
  static bool attr = false;
  if (!attr) {
    ND_CUDA(cudaFuncSetAttribute(sweep9_kernel<T, TC, KIND, OM1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 96 * 1024));
    attr = true;
  }
  if (smem > 96 * 1024) return NDIAG_EINVAL;
  if (P.coupled && !P.paired) {
    // the x-interfaces advance in step: every CTA must be resident
    int per_sm = 0;
    ND_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep9_kernel<T, TC, KIND, OM1>, T9, smem));
    if ((int64_t)per_sm * h->sm_count < (int64_t)nsub) {
      set_error("9-point decomposed sweep: more subdomains than resident CTAs");
      return NDIAG_EINVAL;
    }
    const size_t need = sizeof(unsigned) * nsub;
    if (need > h->sync_bytes) {
      dev_free(h->sync, h->sync_bytes, h->stream);
      h->sync = (unsigned*)dev_alloc(need, h->stream);
      h->sync_bytes = h->sync ? need : 0;
      if (!h->sync) return NDIAG_ENOMEM;
    }
    ND_CUDA(cudaMemsetAsync(h->sync, 0, need, h->stream));
    P.prog = h->sync;
  }
  const int slot = prof_begin(h);
  ++h->launches;
  ++h->sweep_launches;
  sweep9_kernel<T, TC, KIND, OM1><<<nsub, T9, smem, h->stream>>>(P);
  ND_CUDA(cudaGetLastError());
  prof_end(h, slot, bytes);
  return NDIAG_OK;
}

}  // namespace

// Whether a decomposed 9-point sweep with rows of subdomains of height
// ceil(ny / py) keeps its CTAs in step through global memory (subdomains
// taller than a pair CTA's half), and so needs every CTA resident.
bool sweep9_needs_residency(int64_t ny, int py) {
  if (py < 1) return true;
  return (ny + py - 1) / py > T9 / 2;
}

namespace {

template <class T, class TC>
ndiag_status sweep9_t(Handle* h, int kind, int mode, int64_t t, const double* omega, const ScaledSet& set,
                      const void* rhs, const void* xold, void* xnew, double beta_scale) {
  unsigned nsub = 0;
  P9<T, TC> P = params9<T, TC>(h, mode, t, set, rhs, xold, xnew, nsub);
  bool om1 = beta_scale == 1.0;
  for (int k = 0; k < 4; ++k) {
    const double wv = omega ? (mode == NDIAG_DECOMPOSED ? omega[k] : omega[0]) : 1.0;
    P.om[k] = (T)wv;
    if (wv != 1.0) om1 = false;
  }
  P.bscale = (T)beta_scale;
  const double cellbytes = kind == KIND_SOR ? 9.0 * sizeof(TC) + 3.0 * sizeof(T)
                                            : (kind == KIND_TRI_SCALED ? 5.0 : 4.0) * sizeof(TC) + 2.0 * sizeof(T);
  const double bytes = cellbytes * (double)h->N;
  if (kind == KIND_SOR)
    return om1 ? run9<T, TC, KIND_SOR, true>(h, P, nsub, bytes) : run9<T, TC, KIND_SOR, false>(h, P, nsub, bytes);
  if (kind == KIND_TRI_SCALED)
    return om1 ? run9<T, TC, KIND_TRI_SCALED, true>(h, P, nsub, bytes)
               : run9<T, TC, KIND_TRI_SCALED, false>(h, P, nsub, bytes);
  return om1 ? run9<T, TC, KIND_TRI_UNIT, true>(h, P, nsub, bytes)
             : run9<T, TC, KIND_TRI_UNIT, false>(h, P, nsub, bytes);
}

}  // namespace

ndiag_status launch_sweep9(Handle* h, int kind, int mode, int64_t t, const double* omega, const ScaledSet& set,
                           const void* rhs, const void* xold, void* xnew, double beta_scale) {
  // fp64 decomposed triangular sweeps without relaxation: the wavefront kernel
  if (kind != KIND_SOR && !omega && beta_scale == 1.0 && h->precision == NDIAG_FP64 && mode == NDIAG_DECOMPOSED &&
      h->w9_wave) {
    const ndiag_status st = launch_sweep9w(h, kind, mode, t, set, rhs, xnew);
    if (st != NDIAG_EINVAL) return st;
  }
  switch (h->precision) {
    case NDIAG_FP64: return sweep9_t<double, double>(h, kind, mode, t, omega, set, rhs, xold, xnew, beta_scale);
    case NDIAG_FP32: return sweep9_t<float, float>(h, kind, mode, t, omega, set, rhs, xold, xnew, beta_scale);
    default: return sweep9_t<float, __half>(h, kind, mode, t, omega, set, rhs, xold, xnew, beta_scale);
  }
}

ndiag_status launch_ilu_factor9_into(Handle* h, int mode, double* out) {
  unsigned nsub = 0;
  P9<double, double> P = params9<double, double>(h, mode, fwd_phase(2), h->sor, nullptr, nullptr, nullptr, nsub);
  ++h->launches;
  factor9_kernel<<<nsub, T9, 0, h->stream>>>(P, h->A64, out, h->N);
  ND_CUDA(cudaGetLastError());
  return NDIAG_OK;
}

}  // namespace nd
