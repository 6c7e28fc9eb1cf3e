// Decomposed sequential sweep on 3D 7-point matrices (sm_103a), by levels.
//
// In the local frame of a subdomain (reflected so that it sweeps towards +x,
// +y, +z), the paper's 3D sweep (Sec. 4) makes a cell depend on its upstream
// neighbours inside the subdomain, and a cell on a start face whose
// neighbour's subdomain also starts at that face is solved together with it:
// 2x2 systems on faces, 4x4 systems along edges, the 8x8 system at the corner
// (the 3D counterparts of Eqs. 2d:sor2b2 and 2d:sor4b4). With own cell
// (x, y, z) and the set C of coupled axes on which it lies at 0, the block of
// (x, y, z) holds the own cell and its 2^|C| - 1 twins (coordinate -1 on a
// subset of C, i.e. cells of the neighbouring subdomains). Every member's
// upstream neighbours outside the block belong to the blocks of (x-1, y, z),
// (x, y-1, z), (x, y, z-1), so block (x, y, z) can be solved at level
// x + y + z: one CTA per subdomain walks the levels with a block barrier
// between them, one own cell (and its block) per thread.
//
// The CTA recomputes the twins itself (values kept in shared memory) instead
// of waiting for the neighbours; members are ordered canonically (by global
// coordinate along each coupled axis) and every term is formed in a fixed
// order, so all CTAs that solve a block get the same bits.
//
// Transposed solve (D + w L^T) y = v of the SSOR preconditioner: a twin's
// dependents include cells deeper in its own subdomain, so twins cannot be
// recomputed locally in one pass. It runs as four launches in decreasing
// level order: interiors (cells on no coupled start face), then face blocks,
// edge blocks and corner blocks; each reads the earlier launches' results
// from global memory and recomputes only the twins of its own pass.
//
// The decomposed ILU(0) pivots follow d_i = a_ii - sum_{j in J_i, i not in J_j}
// a_ij a_ji / d_j (Sec. 5); mutual pairs drop out, so only upstream cells of
// the same subdomain enter and no twins are needed.
#include <algorithm>

#include "sweep_common.cuh"

namespace nd {
namespace {

using namespace sweep;

constexpr int GT = 256;  // threads per CTA

enum { REG_ALL = 0, REG_INTERIOR = 1, REG_FACES = 2, REG_EDGES = 3, REG_CORNERS = 4, REG_BLOCKS = 5 };

template <class T, class TC>
struct GP {  // 3D only (dim == 3)
  int n[3];
  int64_t stride[3];  // 1, nx, nx * ny
  Split sp[3];
  int dim;
  int base;        // start corner of subdomain (0,0,0): bit a set = starts at max along a
  int coupled;     // interface coupling on (decomposed ordering)
  int transposed;  // (D + w L^T) solve: decreasing levels, dependents instead of predecessors
  int region;      // REG_*
  const TC* inv;
  const TC* c[6];  // scaled entries W E S N B F (transposed entries when transposed)
  const T* rhs;
  const T* xold;
  T* xnew;
  T om[8];  // relaxation per start corner
  T bscale;
  DevStatus* st;
  int twin_slots;  // elements of the twin store
  // forward block records (or null): record q of subdomain s at brec[s * twin_slots + q],
  // q = the twin-store slot of the block's own cell on its first coupled face
  const void* brec;
  // level-ordered copy of the scaled set (or null): array k of subdomain s at
  // level L and row q = y + h0 z of the reference frame is
  // lev[k * lev_arr + s * lev_sub + L * lev_hd0 + q]; lev_flip = axes on which
  // this launch's frame is the reference frame reversed
  const TC* lev;
  int64_t lev_arr, lev_sub;
  int lev_h0, lev_hd0, lev_flip;
};

struct Sub {
  int idx[3], g0[3], len[3], c[3], t[3];
  __device__ int gco(int a, int l) const { return c[a] ? g0[a] + len[a] - 1 - l : g0[a] + l; }
};

// entry index (0-based in c[]) of the neighbour along axis a towards -a / +a
__device__ __forceinline__ int ent(int a, int plus) { return 2 * a + plus; }
// the entry array itself; with a known at compile time both candidates are
// constant indices, so the parameter block need not be copied to local memory
template <class T, class TC>
__device__ __forceinline__ const TC* cptr(const GP<T, TC>& P, int a, int plus) {
  return plus ? P.c[2 * a + 1] : P.c[2 * a];
}
// r-th set bit (axis) of a coupled-axis mask, at compile time
__host__ __device__ constexpr int axis_of(int CM, int r) {
  return r == 0 ? ((CM & 1) ? 0 : (CM & 2) ? 1 : 2) : axis_of(CM & (CM - 1), r - 1);
}

template <class T, class TC>
__device__ __forceinline__ Sub subdomain(const GP<T, TC>& P, unsigned b) {
  Sub S;
  int idx[3];
  idx[0] = (int)(b % (unsigned)P.sp[0].p);
  b /= (unsigned)P.sp[0].p;
  idx[1] = (int)(b % (unsigned)P.sp[1].p);
  idx[2] = (int)(b / (unsigned)P.sp[1].p);
  int cidx = P.base;
  for (int a = 0; a < 3; ++a) {
    S.idx[a] = idx[a];
    S.g0[a] = P.sp[a].lo(idx[a]);
    S.len[a] = P.sp[a].len(idx[a]);
    cidx ^= (idx[a] & 1) << a;
  }
  for (int a = 0; a < 3; ++a) {
    S.c[a] = (cidx >> a) & 1;
    S.t[a] = P.coupled && a < P.dim && (S.c[a] ? S.g0[a] + S.len[a] < P.n[a] : S.g0[a] > 0);
  }
  return S;
}

// Twin store: subset s of {x, y, z} (axes on which the member is at -1), at
// the member's remaining coordinates.
struct TwinIdx {
  int off[8];
  int w, h, d;
  __device__ int slot(int s, const int* lc) const {
    switch (s) {
      case 1: return off[1] + lc[1] * d + lc[2];  // x-face: (y, z)
      case 2: return off[2] + lc[0] * d + lc[2];  // y-face: (x, z)
      case 4: return off[4] + lc[0] * h + lc[1];  // z-face: (x, y)
      case 3: return off[3] + lc[2];              // xy-edge: z
      case 5: return off[5] + lc[1];              // xz-edge: y
      case 6: return off[6] + lc[0];              // yz-edge: x
      default: return off[7];                     // corner
    }
  }
};

__host__ __device__ inline int twin_store_size(int w, int h, int d) { return h * d + w * d + w * h + d + h + w + 1; }

__device__ __forceinline__ TwinIdx twin_index(int w, int h, int d) {
  TwinIdx t;
  t.w = w;
  t.h = h;
  t.d = d;
  t.off[0] = 0;
  t.off[1] = 0;
  t.off[2] = h * d;
  t.off[4] = t.off[2] + w * d;
  t.off[3] = t.off[4] + w * h;
  t.off[5] = t.off[3] + d;
  t.off[6] = t.off[5] + h;
  t.off[7] = t.off[6] + w;
  return t;
}

// Blocks of C = set of coupled axes on which the own cell lies at 0.
__device__ __forceinline__ bool in_region(int region, int C) {
  const int k = __popc(C);
  switch (region) {
    case REG_INTERIOR: return k == 0;
    case REG_FACES: return k == 1;
    case REG_EDGES: return k == 2;
    case REG_CORNERS: return k == 3;
    case REG_BLOCKS: return k > 0;
    default: return true;
  }
}

// One coupled block: the own cell (x, y, z) lies at 0 on the NC coupled axes C.
// Solves the block, stores the own member to xnew and the twins to the twin
// store, and returns the own member's value.
// CM = the coupled axes as a compile-time mask (then C == CM), or 0: taken
// from C at run time. The 4-byte variants use the mask, so that every axis
// index is a constant and no small array lives in local memory; the fp64
// variants keep one instantiation per block size, which holds their code
// and registers down.
template <class T, class TC, int KIND, bool OM1, int NC, int CM = 0>
__device__ __forceinline__ T block_solve(const GP<T, TC>& P, const Sub& S, const TwinIdx& TI, T* tw, int x, int y,
                                      int z, int C, int tcode) {
  const int own[3] = {x, y, z};
  // canonical member order: bit r of a member index <-> r-th coupled axis,
  // set when the member has the larger global coordinate along it
  int axes[3], nC = 0;
  if constexpr (CM != 0) {
    C = CM;
    axes[0] = axis_of(CM, 0);
    axes[1] = NC > 1 ? axis_of(CM, 1) : 0;
    axes[2] = NC > 2 ? axis_of(CM, 2) : 0;
    nC = NC;
  } else {
    for (int a = 0; a < 3; ++a)
      if (C >> a & 1) axes[nC++] = a;
  }
  constexpr int n = 1 << NC;  // nC == NC
  int mo = 0;  // own member
#pragma unroll
  for (int r = 0; r < NC; ++r)
    if (S.c[axes[r]] == 0) mo |= 1 << r;
  T M[n][n], hv[n];
  int64_t gidx[n];
  // coupling of member m to its block partner across each coupled axis
  // (member index m ^ 2^r: constant indices, so M stays in registers)
  auto partners = [&](int m, const int* cm, int64_t gi, T om) {
#pragma unroll
    for (int r = 0; r < NC; ++r) {
      const int a = axes[r];
      T g = ldco<T, TC>(cptr(P, a, cm[a] ? 1 : 0) + gi);
      if (!OM1) g *= om;
      M[m][m ^ (1 << r)] = g;
    }
  };
#pragma unroll
  for (int m = 0; m < n; ++m) {
    int lc[3] = {own[0], own[1], own[2]}, sub = 0;
#pragma unroll
    for (int r = 0; r < NC; ++r)
      if (((m ^ mo) >> r) & 1) {
        lc[axes[r]] = -1;
        sub |= 1 << axes[r];
      }
    int cm[3];
    for (int a = 0; a < 3; ++a) cm[a] = S.c[a] ^ ((sub >> a) & 1);
    int64_t gi = 0;
    int gc[3];
    for (int a = 0; a < 3; ++a) {
      gc[a] = S.gco(a, lc[a]);
      gi += (int64_t)gc[a] * P.stride[a];
    }
    gidx[m] = gi;
    const T om = OM1 ? T(1) : P.om[cm[0] | (cm[1] << 1) | (cm[2] << 2)];
#pragma unroll
    for (int k = 0; k < n; ++k) M[m][k] = T(0);
    M[m][m] = T(1);
    T acc;
    if (!P.transposed) {
      if (KIND == KIND_SOR) {
        T e = ldco<T, TC>(P.inv + gi) * __ldg(P.rhs + gi);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          const int dn = cm[a] ? 0 : 1;  // downstream side of the member along a
          const int gd = gc[a] + (dn ? 1 : -1);
          if (gd >= 0 && gd < P.n[a])
            e = fma(-ldco<T, TC>(cptr(P, a, dn) + gi), __ldg(P.xold + gi + (dn ? P.stride[a] : -P.stride[a])), e);
          const bool implicit_up = (C >> a & 1) || lc[a] >= 1;
          const int gu = gc[a] + (dn ? -1 : 1);
          if (!implicit_up && gu >= 0 && gu < P.n[a])
            e = fma(-ldco<T, TC>(cptr(P, a, 1 - dn) + gi), __ldg(P.xold + gi + (dn ? -P.stride[a] : P.stride[a])), e);
        }
        acc = OM1 ? e : fma(om, e, (T(1) - om) * __ldg(P.xold + gi));
      } else if (KIND == KIND_TRI_SCALED) {
        acc = ldco<T, TC>(P.inv + gi) * __ldg(P.rhs + gi);
        if (!OM1) acc *= P.bscale;
      } else {
        acc = __ldg(P.rhs + gi);
      }
      // upstream neighbours: block partners, or earlier blocks' members.
      // Every load is issued without a branch (absent terms read the member's
      // own cell and are dropped by a select), so that all of a block's loads
      // can be in flight at once.
      partners(m, cm, gi, om);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const int up = cm[a] ? 1 : 0;  // upstream side of the member along a
        const bool use = !(C >> a & 1) && lc[a] >= 1;
        T g = ldco<T, TC>(cptr(P, a, up) + gi);
        if (!OM1) g *= om;
        const int64_t gp = use ? gi + (up ? P.stride[a] : -P.stride[a]) : gi;
        int pc[3] = {lc[0], lc[1], lc[2]};
        pc[a] = use ? pc[a] - 1 : 0;
        const T vg = __ldcg(P.xnew + gp);
        const T vt = sub != 0 ? tw[TI.slot(sub, pc)] : T(0);
        const T v = sub == 0 ? vg : vt;
        acc = use ? fma(-g, v, acc) : acc;
      }
    } else {
      // transposed: dependents are the downstream neighbours inside the
      // member's own subdomain, and the block partners
      acc = __ldg(P.rhs + gi);
      partners(m, cm, gi, om);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const int up = cm[a] ? 1 : 0, dn = 1 - up;
        // downstream neighbour inside the member's subdomain: local
        // coordinate +1 (own side), or -2 (twin side along a)
        const bool twin_axis = (sub >> a) & 1;
        const int gd = gc[a] + (dn ? 1 : -1);
        bool inside;
        if (twin_axis) {  // the twin's subdomain: the neighbour across S's start face
          const int it = S.c[a] ? S.idx[a] + 1 : S.idx[a] - 1;
          const int t0 = P.sp[a].lo(it), t1 = t0 + P.sp[a].len(it);
          inside = gd >= t0 && gd < t1;
        } else {
          inside = lc[a] + 1 < S.len[a];
        }
        // loads without a branch, as in the forward case
        T g = ldco<T, TC>(cptr(P, a, dn) + gi);
        if (!OM1) g *= om;
        const int64_t gq = inside ? gi + (dn ? P.stride[a] : -P.stride[a]) : gi;
        // same twin subset one step downstream: this launch's store if that
        // block is of the same kind, else an earlier launch
        int pc[3] = {lc[0], lc[1], lc[2]};
        pc[a] += 1;
        int oc[3] = {own[0], own[1], own[2]};
        oc[a] += 1;
        const int C2 = ((oc[0] == 0) | ((oc[1] == 0) << 1) | ((oc[2] == 0) << 2)) & tcode;
        const bool from_tw = inside && !(sub == 0 || twin_axis) && __popc(C2) == nC;
        if (!from_tw) pc[0] = pc[1] = pc[2] = 0;
        const T vg = __ldcg(P.xnew + gq);
        const T vt = sub != 0 ? tw[TI.slot(sub, pc)] : T(0);
        const T v = from_tw ? vt : vg;
        acc = inside ? fma(-g, v, acc) : acc;
      }
    }
    hv[m] = acc;
  }
  // (I + G) x = h, elimination in canonical order (diagonally dominant: no pivoting)
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
      int lc[3] = {own[0], own[1], own[2]}, sub = 0;
#pragma unroll
      for (int r = 0; r < NC; ++r)
        if (((m ^ mo) >> r) & 1) {
          lc[axes[r]] = -1;
          sub |= 1 << axes[r];
        }
      tw[TI.slot(sub, lc)] = xs[m];
    }
  }
  T own_x = xs[0];
#pragma unroll
  for (int m = 1; m < n; ++m)
    if (m == mo) own_x = xs[m];
  return own_x;
}

// Record of one coupled face or edge block (2 or 4 members) of a forward
// pass, in the members' canonical order: everything of block_solve's forward
// branch that depends neither on the right-hand side nor on new values --
// member cells, pivots, the upstream couplings and where their values come
// from, and the inverse of the block matrix (Gauss-Jordan in the canonical
// order, so that every CTA solving the block holds the same inverse). A solve
// is then a gather and a small matrix-vector product.
constexpr int64_t BREC_NONE = INT64_MIN;

template <class T>
struct BRec {
  int64_t gi[4];      // member cells
  int64_t src[4][3];  // upstream value: >= 0 a cell of xnew, < 0 the twin slot -1 - src, BREC_NONE absent
  T inv[4];
  T g[4][3];          // upstream couplings (0 where absent)
  T minv[16];         // n x n, row-major
  int dst[4];         // -1: the own member (to xnew), else its twin slot
  int n, own;
};

template <class T, class TC, int KIND, int NC, bool TR>
__device__ void block_record(const GP<T, TC>& P, const Sub& S, const TwinIdx& TI, int x, int y, int z, int C,
                             int tcode, BRec<T>& R) {
  const int own[3] = {x, y, z};
  int axes[3] = {0, 0, 0}, nC = 0;
  for (int a = 0; a < 3; ++a)
    if (C >> a & 1) axes[nC++] = a;
  constexpr int n = 1 << NC;
  int mo = 0;
  for (int r = 0; r < NC; ++r)
    if (S.c[axes[r]] == 0) mo |= 1 << r;
  double M[n][n];
  R.n = n;
  R.own = mo;
  for (int m = 0; m < n; ++m) {
    int lc[3] = {own[0], own[1], own[2]}, sub = 0;
    for (int r = 0; r < NC; ++r)
      if (((m ^ mo) >> r) & 1) {
        lc[axes[r]] = -1;
        sub |= 1 << axes[r];
      }
    int cm[3];
    for (int a = 0; a < 3; ++a) cm[a] = S.c[a] ^ ((sub >> a) & 1);
    int64_t gi = 0;
    for (int a = 0; a < 3; ++a) gi += (int64_t)S.gco(a, lc[a]) * P.stride[a];
    R.gi[m] = gi;
    R.inv[m] = (!TR && KIND == KIND_TRI_SCALED) ? ldco<T, TC>(P.inv + gi) : T(0);
    R.dst[m] = sub == 0 ? -1 : TI.slot(sub, lc);
    for (int k = 0; k < n; ++k) M[m][k] = k == m ? 1.0 : 0.0;
    for (int r = 0; r < NC; ++r) {
      const int a = axes[r];
      M[m][m ^ (1 << r)] = (double)ldco<T, TC>(cptr(P, a, cm[a] ? 1 : 0) + gi);
    }
    for (int a = 0; a < 3; ++a) {
      const int up = cm[a] ? 1 : 0;
      if (!TR) {  // upstream neighbours of the member (block_solve's forward branch)
        const bool use = !(C >> a & 1) && lc[a] >= 1;
        R.g[m][a] = use ? ldco<T, TC>(cptr(P, a, up) + gi) : T(0);
        if (!use) {
          R.src[m][a] = BREC_NONE;
        } else if (sub == 0) {
          R.src[m][a] = gi + (up ? P.stride[a] : -P.stride[a]);
        } else {
          int pc[3] = {lc[0], lc[1], lc[2]};
          pc[a] -= 1;
          R.src[m][a] = -1 - (int64_t)TI.slot(sub, pc);
        }
      } else {  // downstream dependents inside the member's subdomain (the transposed branch)
        const int dn = 1 - up;
        const bool twin_axis = (sub >> a) & 1;
        const int gd = S.gco(a, lc[a]) + (dn ? 1 : -1);
        bool inside;
        if (twin_axis) {
          const int it = S.c[a] ? S.idx[a] + 1 : S.idx[a] - 1;
          const int t0 = P.sp[a].lo(it), t1 = t0 + P.sp[a].len(it);
          inside = gd >= t0 && gd < t1;
        } else {
          inside = lc[a] + 1 < S.len[a];
        }
        R.g[m][a] = inside ? ldco<T, TC>(cptr(P, a, dn) + gi) : T(0);
        if (!inside) {
          R.src[m][a] = BREC_NONE;
          continue;
        }
        const int64_t gq = gi + (dn ? P.stride[a] : -P.stride[a]);
        int pc[3] = {lc[0], lc[1], lc[2]};
        pc[a] += 1;
        int oc[3] = {own[0], own[1], own[2]};
        oc[a] += 1;
        const int C2 = ((oc[0] == 0) | ((oc[1] == 0) << 1) | ((oc[2] == 0) << 2)) & tcode;
        const bool from_tw = !(sub == 0 || twin_axis) && __popc(C2) == NC;
        R.src[m][a] = from_tw ? -1 - (int64_t)TI.slot(sub, pc) : gq;
      }
    }
  }
  for (int m = n; m < 4; ++m) {
    R.gi[m] = R.gi[0];
    R.inv[m] = T(0);
    R.dst[m] = -1;
    for (int a = 0; a < 3; ++a) {
      R.g[m][a] = T(0);
      R.src[m][a] = BREC_NONE;
    }
  }
  // inverse by Gauss-Jordan (diagonally dominant: no pivoting), in fp64
  double I[n][n];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) I[i][j] = i == j ? 1.0 : 0.0;
  for (int k = 0; k < n; ++k) {
    const double r = 1.0 / M[k][k];
    for (int j = 0; j < n; ++j) {
      M[k][j] *= r;
      I[k][j] *= r;
    }
    for (int i = 0; i < n; ++i) {
      if (i == k) continue;
      const double f = M[i][k];
      for (int j = 0; j < n; ++j) {
        M[i][j] = fma(-f, M[k][j], M[i][j]);
        I[i][j] = fma(-f, I[k][j], I[i][j]);
      }
    }
  }
  for (int i = 0; i < 16; ++i) R.minv[i] = T(0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) R.minv[i * n + j] = (T)I[i][j];
}

// The forward solve of a recorded block: h_m = pivot r - sum of the upstream
// terms (in the order of block_solve), x = Minv h; the own member to xnew, the
// twins to the twin store.
template <class T, class TC, int KIND, int N>
__device__ __forceinline__ void block_solve_rec(const GP<T, TC>& P, const BRec<T>* __restrict__ R, T* tw) {
  T hv[N];
#pragma unroll
  for (int m = 0; m < N; ++m) {
    const int64_t gi = __ldg(&R->gi[m]);
    const T rr = __ldg(P.rhs + gi);
    T acc = KIND == KIND_TRI_SCALED ? __ldg(&R->inv[m]) * rr : rr;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      // absent terms read the member's own cell and are dropped by a select
      // (that value may be anything, even not a number)
      const int64_t sr = __ldg(&R->src[m][a]);
      const bool use = sr != BREC_NONE;
      const int64_t sc = use ? sr : gi;
      const T vg = __ldcg(P.xnew + (sc >= 0 ? sc : gi));
      const T vt = tw[sc >= 0 ? 0 : (int)(-1 - sc)];
      const T v = sc >= 0 ? vg : vt;
      acc = use ? fma(-__ldg(&R->g[m][a]), v, acc) : acc;
    }
    hv[m] = acc;
  }
#pragma unroll
  for (int i = 0; i < N; ++i) {
    T xs = T(0);
#pragma unroll
    for (int j = 0; j < N; ++j) xs = fma(__ldg(&R->minv[i * N + j]), hv[j], xs);
    const int dd = __ldg(&R->dst[i]);
    if (dd < 0) P.xnew[__ldg(&R->gi[i])] = xs;
    else tw[dd] = xs;
  }
}

// Builds the forward block records of one phase: one thread per (subdomain,
// twin-store slot); slots that hold no face or edge block of the forward pass
// get n = 0.
template <class T, class TC, int KIND, bool TR>
__global__ void block_record_kernel(GP<T, TC> P, BRec<T>* out, int64_t total) {
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const unsigned sb = (unsigned)(q / P.twin_slots);
    const int slot = (int)(q % P.twin_slots);
    const Sub S = subdomain(P, sb);
    const int w = S.len[0], h = S.len[1], d = S.len[2];
    const TwinIdx TI = twin_index(w, h, d);
    const int tcode = S.t[0] | (S.t[1] << 1) | (S.t[2] << 2);
    BRec<T> R;
    R.n = 0;
    int x = -1, y = -1, z = -1, a = -1;
    if (slot < TI.off[2]) {
      a = 0, x = 0, y = slot / d, z = slot % d;
    } else if (slot < TI.off[4]) {
      a = 1, y = 0, x = (slot - TI.off[2]) / d, z = (slot - TI.off[2]) % d;
    } else if (slot < TI.off[3]) {
      a = 2, z = 0, x = (slot - TI.off[4]) / h, y = (slot - TI.off[4]) % h;
    }
    if (a >= 0 && x < w && y < h && z < d) {
      const int own[3] = {x, y, z};
      const int C = ((x == 0) | ((y == 0) << 1) | ((z == 0) << 2)) & tcode;
      int first = -1;
      for (int b = 0; b < 3; ++b)
        if (first < 0 && ((C >> b) & 1) && own[b] == 0) first = b;
      if (first == a) {
        if (__popc(C) == 1) block_record<T, TC, KIND, 1, TR>(P, S, TI, x, y, z, C, tcode, R);
        else if (__popc(C) == 2) block_record<T, TC, KIND, 2, TR>(P, S, TI, x, y, z, C, tcode, R);
      }
    }
    out[q] = R;
  }
}

// the 8x8 corner block (one per subdomain) of the fp64 variants out of line,
// so that its registers do not weigh on the face and edge blocks
template <class T, class TC, int KIND, bool OM1>
__device__ __noinline__ void corner_block(const GP<T, TC>& P, const Sub& S, const TwinIdx& TI, T* tw, int x, int y,
                                          int z, int C, int tcode) {
  block_solve<T, TC, KIND, OM1, 3>(P, S, TI, tw, x, y, z, C, tcode);
}

// the 8x8 corner of the 4-byte variants out of line in the six-warp block
// kernel, so that it does not set that kernel's register budget
template <class T, class TC, int KIND, bool OM1>
__device__ __noinline__ void corner_block_cm(const GP<T, TC>& P, const Sub& S, const TwinIdx& TI, T* tw, int x,
                                             int y, int z, int C, int tcode) {
  block_solve<T, TC, KIND, OM1, 3, 7>(P, S, TI, tw, x, y, z, C, tcode);
}

// One level walk of a subdomain. SIX: the block passes of subdomains up to 32
// a side in six warps (4-byte variants): warps 0..2 take the cells of the x,
// y and z faces, lane 0 of warps 3..5 those of the xy, xz and yz edges (warp
// 3 also the corner). Every warp then runs one block solve with compile-time
// axes, and the three edges' 4x4 systems run side by side.
template <class T, class TC, int KIND, bool OM1, bool SIX>
__device__ __forceinline__ void sweep3d_body(const GP<T, TC>& P) {
  extern __shared__ __align__(16) unsigned char gsm[];
  T* tw = reinterpret_cast<T*>(gsm);
  const Sub S = subdomain(P, blockIdx.x);
  const int w = S.len[0], h = S.len[1], d = S.len[2];
  const TwinIdx TI = twin_index(w, h, d);
  const int lmax = (w - 1) + (h - 1) + (d - 1);
  const int tcode = S.t[0] | (S.t[1] << 1) | (S.t[2] << 2);
  const bool blocks_only = P.region != REG_ALL && P.region != REG_INTERIOR;
  const int umax = max(w, max(h, d));
  // block cells lie on start faces: a face cell (two free coordinates) is on
  // a level <= 2 (umax - 1), an edge cell (one) on a level <= umax - 1, the
  // corner on level 0; the passes over blocks skip the empty levels above
  const int lreg = P.region == REG_CORNERS ? 0
                   : P.region == REG_EDGES ? min(lmax, umax - 1)
                   : blocks_only           ? min(lmax, 2 * (umax - 1))
                                           : lmax;
  for (int it = 0; it <= lreg; ++it) {
    const int L = P.transposed ? lreg - it : it;
    // REG_ALL / REG_INTERIOR: every row (y, z) meets its cell x = L - y - z.
    // Block regions: only cells with a zero coordinate can be blocks; cell c
    // of a level enumerates face a = c / umax (coordinate a = 0), the cell
    // taken on the first face where it has a zero coordinate.
    // Without SIX (8-byte variants, 4 warps): warps 0..2 the faces, lanes
    // 0..2 of warp 3 the edges, through the solve with run-time axes (one
    // code path, so the three edges still run side by side).
    const bool split = SIX || (blocks_only && umax <= 32);
    const int nq = SIX ? 6 * 32 : split ? 4 * 32 : blocks_only ? 3 * umax : h * d;
    for (int q = threadIdx.x; q < nq; q += blockDim.x) {
      int x, y, z;
      if (!blocks_only) {
        y = q % h;
        z = q / h;
        x = L - y - z;
        if (x < 0 || x >= w) continue;
      } else if (split && q >= 3 * 32) {
        const int e = SIX ? (q - 3 * 32) >> 5 : q - 3 * 32;
        if ((SIX && (q & 31) != 0) || e >= 3 || (L == 0 && e > 0)) continue;
        x = e == 2 ? L : 0;
        y = e == 1 ? L : 0;
        z = e == 0 ? L : 0;
        if (x >= w || y >= h || z >= d) continue;
        const int Ce = ((x == 0) | ((y == 0) << 1) | ((z == 0) << 2)) & tcode;
        if (__popc(Ce) < 2) continue;  // a face cell (its face warp takes it) or none
      } else {
        const int a = split ? q >> 5 : q / umax, u = split ? q & 31 : q - a * umax;
        const int lu = a == 0 ? h : w, lv = a == 2 ? h : d;
        const int v = L - u;
        if (u >= lu || v < 0 || v >= lv) continue;
        if (a == 0) {
          x = 0, y = u, z = v;
        } else if (a == 1) {
          x = u, y = 0, z = v;
          if (x == 0) continue;
        } else {
          x = u, y = v, z = 0;
          if (x == 0 || y == 0) continue;
        }
        if (split && __popc(((x == 0) | ((y == 0) << 1) | ((z == 0) << 2)) & tcode) >= 2) continue;  // an edge warp's
      }
      const int own[3] = {x, y, z};
      const int C = ((x == 0) | ((y == 0) << 1) | ((z == 0) << 2)) & tcode;
      if (!in_region(P.region, C)) continue;
      if (C == 0) {  // a block of one cell
        int64_t gi = 0;
        int gc[3];
        for (int a = 0; a < 3; ++a) {
          gc[a] = S.gco(a, own[a]);
          gi += (int64_t)gc[a] * P.stride[a];
        }
        const T om = OM1 ? T(1) : P.om[S.c[0] | (S.c[1] << 1) | (S.c[2] << 2)];
        T acc;
        if (!P.transposed) {
          if (KIND == KIND_SOR) {
            T e = ldco<T, TC>(P.inv + gi) * __ldg(P.rhs + gi);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
              const int dn = S.c[a] ? 0 : 1;
              const int gd = gc[a] + (dn ? 1 : -1);
              if (gd >= 0 && gd < P.n[a])
                e = fma(-ldco<T, TC>(cptr(P, a, dn) + gi), __ldg(P.xold + gi + (dn ? P.stride[a] : -P.stride[a])), e);
              const int gu = gc[a] + (dn ? -1 : 1);
              if (own[a] == 0 && gu >= 0 && gu < P.n[a])
                e = fma(-ldco<T, TC>(cptr(P, a, 1 - dn) + gi), __ldg(P.xold + gi + (dn ? -P.stride[a] : P.stride[a])), e);
            }
            acc = OM1 ? e : fma(om, e, (T(1) - om) * __ldg(P.xold + gi));
          } else if (KIND == KIND_TRI_SCALED) {
            acc = ldco<T, TC>(P.inv + gi) * __ldg(P.rhs + gi);
            if (!OM1) acc *= P.bscale;
          } else {
            acc = __ldg(P.rhs + gi);
          }
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            if (own[a] < 1) continue;
            const int up = S.c[a] ? 1 : 0;
            T g = ldco<T, TC>(cptr(P, a, up) + gi);
            if (!OM1) g *= om;
            acc = fma(-g, __ldcg(P.xnew + gi + (up ? P.stride[a] : -P.stride[a])), acc);
          }
        } else {
          acc = __ldg(P.rhs + gi);
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            if (own[a] + 1 >= S.len[a]) continue;
            const int dn = S.c[a] ? 0 : 1;
            T g = ldco<T, TC>(cptr(P, a, dn) + gi);
            if (!OM1) g *= om;
            acc = fma(-g, __ldcg(P.xnew + gi + (dn ? P.stride[a] : -P.stride[a])), acc);
          }
        }
        P.xnew[gi] = acc;
        continue;
      }
      if (P.brec && (__popc(C) == 1 || __popc(C) == 2)) {  // a recorded block
        const int f = (own[0] == 0 && (C & 1)) ? 0 : ((own[1] == 0 && (C & 2)) ? 1 : 2);
        const BRec<T>* R = reinterpret_cast<const BRec<T>*>(P.brec) + (int64_t)blockIdx.x * P.twin_slots +
                           TI.slot(1 << f, own);
        if (__popc(C) == 1) block_solve_rec<T, TC, KIND, 2>(P, R, tw);
        else block_solve_rec<T, TC, KIND, 4>(P, R, tw);
        continue;
      }
      if (SIX && __popc(C) == 3) {
        if constexpr (sizeof(T) == 4) corner_block_cm<T, TC, KIND, OM1>(P, S, TI, tw, x, y, z, C, tcode);
        else corner_block<T, TC, KIND, OM1>(P, S, TI, tw, x, y, z, C, tcode);
        continue;
      }
      if (!SIX && split && __popc(C) == 2) {  // the edge warp: one code path for the three edges
        block_solve<T, TC, KIND, OM1, 2>(P, S, TI, tw, x, y, z, C, tcode);
        continue;
      }
      if constexpr (sizeof(T) == 4) {
        switch (C) {  // the coupled axes as a compile-time mask
          case 1: block_solve<T, TC, KIND, OM1, 1, 1>(P, S, TI, tw, x, y, z, C, tcode); break;
          case 2: block_solve<T, TC, KIND, OM1, 1, 2>(P, S, TI, tw, x, y, z, C, tcode); break;
          case 4: block_solve<T, TC, KIND, OM1, 1, 4>(P, S, TI, tw, x, y, z, C, tcode); break;
          case 3: block_solve<T, TC, KIND, OM1, 2, 3>(P, S, TI, tw, x, y, z, C, tcode); break;
          case 5: block_solve<T, TC, KIND, OM1, 2, 5>(P, S, TI, tw, x, y, z, C, tcode); break;
          case 6: block_solve<T, TC, KIND, OM1, 2, 6>(P, S, TI, tw, x, y, z, C, tcode); break;
          default: block_solve<T, TC, KIND, OM1, 3, 7>(P, S, TI, tw, x, y, z, C, tcode);
        }
      } else {
        if (__popc(C) == 1) block_solve<T, TC, KIND, OM1, 1>(P, S, TI, tw, x, y, z, C, tcode);
        else if (__popc(C) == 2) block_solve<T, TC, KIND, OM1, 2>(P, S, TI, tw, x, y, z, C, tcode);
        else corner_block<T, TC, KIND, OM1>(P, S, TI, tw, x, y, z, C, tcode);
      }
    }
    __syncthreads();
  }
}

template <class T, class TC, int KIND, bool OM1>
__global__ void __launch_bounds__(GT, 2) sweep3d_kernel(GP<T, TC> P) {
  sweep3d_body<T, TC, KIND, OM1, false>(P);
}

template <class T, class TC, int KIND, bool OM1>
__global__ void __launch_bounds__(6 * 32, 4) sweep3d_blocks_kernel(GP<T, TC> P) {
  sweep3d_body<T, TC, KIND, OM1, true>(P);
}

// Pencil form of the level walk over the cells of one-cell blocks (C = 0) for
// the triangular kinds (ILU(0) forward and backward, the SSOR forward half,
// and the interior pass of the transposed solve). Thread t owns the rows
// q = t + GT k, i.e. (y, z) = (q mod h, q / h), and meets each row's next cell
// on every level, so
//  * the row's previous cell (x - 1, or x + 1 when transposed) is in a register,
//  * the neighbours along y and z were put into a shared two-level buffer on
//    the level before,
//  * every operand of the next level's cells is loaded before this level's
//    arithmetic starts (one level of prefetch).
// In a forward pass the coupled blocks on the start faces depend only on each
// other, so an earlier launch (sweep3d_kernel over REG_BLOCKS) solves them;
// here their own-cell values are read back from xnew like operands. The
// arithmetic of a cell is the same, operation for operation, as in
// sweep3d_kernel.
constexpr int KR = 4;  // rows per thread: h * d <= KR * GT

template <class T, class TC, int KIND, bool OM1>
__global__ void __launch_bounds__(GT, 4) sweep3d_pencil_kernel(GP<T, TC> P) {
  extern __shared__ __align__(16) unsigned char gsm[];
  T* lv = reinterpret_cast<T*>(gsm);  // [2][hd]: the values of the last two levels, by row
  const Sub S = subdomain(P, blockIdx.x);
  const int w = S.len[0], h = S.len[1], d = S.len[2], hd = h * d;
  const int lmax = (w - 1) + (h - 1) + (d - 1);
  const int tcode = S.t[0] | (S.t[1] << 1) | (S.t[2] << 2);
  const bool tr = P.transposed != 0;
  const T om = OM1 ? T(1) : P.om[S.c[0] | (S.c[1] << 1) | (S.c[2] << 2)];
  int yk[KR], zk[KR];
#pragma unroll
  for (int k = 0; k < KR; ++k) {
    const int q = threadIdx.x + GT * k;
    yk[k] = q < hd ? q % h : 0;
    zk[k] = q < hd ? q / h : 0;
  }
  // global index of the row's cell at local x
  auto gidx = [&](int k, int x) -> int64_t {
    return (int64_t)S.gco(0, x) + (int64_t)S.gco(1, yk[k]) * P.stride[1] + (int64_t)S.gco(2, zk[k]) * P.stride[2];
  };
  // raw operands of each row's cell on the coming level: inv, rhs, and the
  // couplings along x, y, z (0 where the neighbour is absent)
  T pi[KR], pr[KR], pg[KR][3];
  auto fetch = [&](int L) {
#pragma unroll
    for (int k = 0; k < KR; ++k) {
      const int q = threadIdx.x + GT * k;
      const int x = L - yk[k] - zk[k];
      if (q >= hd || x < 0 || x >= w) continue;
      const int C = ((x == 0) | ((yk[k] == 0) << 1) | ((zk[k] == 0) << 2)) & tcode;
      const int64_t gi = gidx(k, x);
      if (C != 0) {  // solved by the block launch (forward passes only)
        if (!tr) pr[k] = __ldcg(P.xnew + gi);
        continue;
      }
      const int own[3] = {x, yk[k], zk[k]};
      // coefficient k of this cell: the level-ordered copy (consecutive rows
      // at consecutive addresses) or the natural arrays
      const TC* cbase;
      int64_t ci;
      if (P.lev) {
        const int xr = (P.lev_flip & 1) ? w - 1 - x : x;
        const int yr = (P.lev_flip & 2) ? h - 1 - yk[k] : yk[k];
        const int zr = (P.lev_flip & 4) ? d - 1 - zk[k] : zk[k];
        cbase = P.lev + (int64_t)blockIdx.x * P.lev_sub;
        ci = (int64_t)(xr + yr + zr) * P.lev_hd0 + yr + P.lev_h0 * zr;
      } else {
        cbase = P.inv;
        ci = gi;
      }
      const int64_t ca = P.lev ? P.lev_arr : (int64_t)(P.c[0] - P.inv);
      if (!tr && KIND == KIND_TRI_SCALED) pi[k] = ldco<T, TC>(cbase + ci);
      pr[k] = __ldg(P.rhs + gi);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        if (!tr) {
          const int up = S.c[a] ? 1 : 0;
          pg[k][a] = own[a] >= 1 ? ldco<T, TC>(cbase + (1 + ent(a, up)) * ca + ci) : T(0);
        } else {
          const int dn = S.c[a] ? 0 : 1;
          pg[k][a] = own[a] + 1 < S.len[a] ? ldco<T, TC>(cbase + (1 + ent(a, dn)) * ca + ci) : T(0);
        }
      }
    }
  };
  T xr[KR];
#pragma unroll
  for (int k = 0; k < KR; ++k) xr[k] = T(0);
  fetch(tr ? lmax : 0);
  for (int it = 0; it <= lmax; ++it) {
    const int L = tr ? lmax - it : it;
    const int cur = it & 1, prv = cur ^ 1;
    T ci[KR], cr[KR], cg[KR][3];
#pragma unroll
    for (int k = 0; k < KR; ++k) {
      ci[k] = pi[k];
      cr[k] = pr[k];
#pragma unroll
      for (int a = 0; a < 3; ++a) cg[k][a] = pg[k][a];
    }
    if (it < lmax) fetch(tr ? L - 1 : L + 1);
#pragma unroll
    for (int k = 0; k < KR; ++k) {
      const int q = threadIdx.x + GT * k;
      const int x = L - yk[k] - zk[k];
      if (q >= hd || x < 0 || x >= w) continue;
      const int C = ((x == 0) | ((yk[k] == 0) << 1) | ((zk[k] == 0) << 2)) & tcode;
      if (C != 0 && tr) continue;  // the transposed block passes follow this one
      T v;
      if (C != 0) {
        v = cr[k];
      } else {
        T acc;
        if (!tr && KIND == KIND_TRI_SCALED) {
          acc = ci[k] * cr[k];
          if (!OM1) acc *= P.bscale;
        } else {
          acc = cr[k];
        }
        T g0 = cg[k][0], g1 = cg[k][1], g2 = cg[k][2];
        if (!OM1) {
          g0 *= om;
          g1 *= om;
          g2 *= om;
        }
        if (!tr) {
          if (x >= 1) acc = fma(-g0, xr[k], acc);
          if (yk[k] >= 1) acc = fma(-g1, lv[prv * hd + q - 1], acc);
          if (zk[k] >= 1) acc = fma(-g2, lv[prv * hd + q - h], acc);
        } else {
          if (x + 1 < w) acc = fma(-g0, xr[k], acc);
          if (yk[k] + 1 < h) acc = fma(-g1, lv[prv * hd + q + 1], acc);
          if (zk[k] + 1 < d) acc = fma(-g2, lv[prv * hd + q + h], acc);
        }
        P.xnew[gidx(k, x)] = acc;
        v = acc;
      }
      lv[cur * hd + q] = v;
      xr[k] = v;
    }
    __syncthreads();
  }
}

// Wavefront form of the pencil walk (subdomains with h, d <= 32): warp z owns
// the plane z and lane y its row y, and at step s lane y meets column
// x = s - y. The x neighbour is the lane's previous cell (register), the y
// neighbour arrives by shuffle from lane y - 1 (its previous step), the z
// neighbour from warp z - 1 through a ring of a few steps in shared memory
// (full / empty mbarriers per chunk, all 32 lanes arriving). A warp runs one
// chunk behind the warp below it, so the walk takes about (w + h + d) chunks'
// worth of steps instead of w + h + d block barriers. The transposed pass runs
// the same walk in the reflected frame (dependents instead of predecessors).
// Operands of the next chunk are loaded before the current one is computed;
// the arithmetic of a cell is that of sweep3d_pencil_kernel.
template <class T>
struct WvCfg {
  static constexpr int CH = 2;                        // steps per chunk (register double buffer)
  static constexpr int R = sizeof(T) == 8 ? 8 : 16;   // ring slots (steps)
  static constexpr int NS = R / CH;                   // ring stages
};

template <class T, class TC, int KIND, bool OM1>
__global__ void __launch_bounds__(1024) sweep3d_wave_kernel(GP<T, TC> P) {
  constexpr int CH = WvCfg<T>::CH, NS = WvCfg<T>::NS, WV_R = WvCfg<T>::R;
  extern __shared__ __align__(16) unsigned char gsm[];
  const Sub S = subdomain(P, blockIdx.x);
  const int w = S.len[0], h = S.len[1], d = S.len[2];
  const int nw = blockDim.x >> 5;
  T* ring = reinterpret_cast<T*>(gsm);  // [nw][WV_R][32]
  unsigned long long* full = reinterpret_cast<unsigned long long*>(gsm + sizeof(T) * (size_t)nw * WV_R * 32);
  unsigned long long* empty = full + nw * NS;
  if (threadIdx.x == 0) {
    for (int i = 0; i < 2 * nw * NS; ++i) mb_init(&full[i], 32);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const int wz = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (wz >= d) return;
  const bool tr = P.transposed != 0;
  const bool row_on = lane < h;
  const int y = tr ? h - 1 - lane : lane, z = tr ? d - 1 - wz : wz;
  const int yc = row_on ? y : 0;
  const int tcode = S.t[0] | (S.t[1] << 1) | (S.t[2] << 2);
  const T om = OM1 ? T(1) : P.om[S.c[0] | (S.c[1] << 1) | (S.c[2] << 2)];
  const int64_t rowbase = (int64_t)S.gco(1, yc) * P.stride[1] + (int64_t)S.gco(2, z) * P.stride[2];
  const int yr = (P.lev_flip & 2) ? h - 1 - yc : yc, zr = (P.lev_flip & 4) ? d - 1 - z : z;
  const int64_t ca = P.lev ? P.lev_arr : (int64_t)(P.c[0] - P.inv);
  const int nsteps = w + h - 1, nch = (nsteps + CH - 1) / CH;
  // Per-lane operand pointers at column xq = 0 of the walk and their step
  // along it: the natural index moves by +-1, the level-ordered one by
  // +-h0 d0 (one level) per column.
  const int x0 = tr ? w - 1 : 0;
  const int64_t gi0 = rowbase + S.gco(0, x0);
  const int dgi = (S.gco(0, x0 + (tr ? -1 : 1)) - S.gco(0, x0));
  const T* prhs = P.rhs + gi0;
  const T* pxn = P.xnew + gi0;
  int64_t ci0;
  int dci;
  if (P.lev) {
    const int xr0 = (P.lev_flip & 1) ? w - 1 - x0 : x0;
    ci0 = (int64_t)blockIdx.x * P.lev_sub + (int64_t)(xr0 + yr + zr) * P.lev_hd0 + yr + P.lev_h0 * zr;
    const int xr1 = (P.lev_flip & 1) ? w - 1 - (x0 + (tr ? -1 : 1)) : x0 + (tr ? -1 : 1);
    dci = (xr1 - xr0) * P.lev_hd0;
  } else {
    ci0 = gi0;
    dci = dgi;
  }
  const TC* cb = (P.lev ? P.lev : P.inv) + ci0;
  const TC* pinv = cb;
  const TC* pg0 = cb + (1 + ent(0, (S.c[0] ^ tr) ? 1 : 0)) * ca;
  const TC* pg1 = cb + (1 + ent(1, (S.c[1] ^ tr) ? 1 : 0)) * ca;
  const TC* pg2 = cb + (1 + ent(2, (S.c[2] ^ tr) ? 1 : 0)) * ca;
  // neighbours along y and z exist for the whole row; along x from column 1 on
  const bool has_y = lane >= 1, has_z = wz > 0;
  // coupled cells: the whole row (a coupled start face in y or z), or column 0 of the walk (in x)
  const bool row_blk = (((y == 0) << 1 | (z == 0) << 2) & tcode) != 0;
  const int xq_blk = (tcode & 1) ? (tr ? w - 1 : 0) : -1;  // walk column of the x-start face, if coupled
  // operands of a chunk: inv, rhs (or the block's value), couplings x, y, z;
  // cur is computed while nxt is loaded
  struct Ops {
    T i[CH], r[CH], g[3][CH];
    unsigned blk;
  };
  auto fetch = [&](int k, Ops& o) {
    o.blk = 0;
#pragma unroll
    for (int j = 0; j < CH; ++j) {
      const int xq = k * CH + j - lane;  // column in the walk's frame
      o.i[j] = T(0);
      o.r[j] = T(0);
      o.g[0][j] = o.g[1][j] = o.g[2][j] = T(0);
      if (!row_on || xq < 0 || xq >= w) continue;
      if (row_blk || xq == xq_blk) {  // a coupled block: the block launch's value (forward), or left to later passes
        o.blk |= 1u << j;
        if (!tr) o.r[j] = __ldcg(pxn + xq * dgi);
        continue;
      }
      const int oc = xq * dci;
      if (!tr && KIND == KIND_TRI_SCALED) o.i[j] = ldco<T, TC>(pinv + oc);
      o.r[j] = __ldg(prhs + xq * dgi);
      if (xq >= 1) o.g[0][j] = ldco<T, TC>(pg0 + oc);
      if (has_y) o.g[1][j] = ldco<T, TC>(pg1 + oc);
      if (has_z) o.g[2][j] = ldco<T, TC>(pg2 + oc);
    }
  };
  T* ring_out = ring + (size_t)wz * WV_R * 32;
  const T* ring_in = ring + (size_t)(wz > 0 ? wz - 1 : 0) * WV_R * 32;
  const bool has_in = wz > 0, has_out = wz + 1 < d;
  bool ok = true;
  T xp = T(0);
  Ops cur, nxt;
  fetch(0, nxt);
  for (int k = 0; k < nch; ++k) {
    cur = nxt;
    if (k + 1 < nch) fetch(k + 1, nxt);
    const int st = k % NS;
    if (has_in && ok) ok = mb_wait(&full[(wz - 1) * NS + st], (k / NS) & 1, P.st);
    if (has_out && ok && k >= NS) ok = mb_wait(&empty[wz * NS + st], ((k / NS) - 1) & 1, P.st);
    if (!ok) return;
#pragma unroll
    for (int j = 0; j < CH; ++j) {
      const int s = k * CH + j, xq = s - lane;
      const T sh = __shfl_up_sync(FULL, xp, 1);
      const bool act = row_on && xq >= 0 && xq < w;
      T v;
      if ((cur.blk >> j) & 1) {
        v = cur.r[j];
      } else {
        T acc = (!tr && KIND == KIND_TRI_SCALED) ? cur.i[j] * cur.r[j] : cur.r[j];
        if (!OM1 && !tr && KIND == KIND_TRI_SCALED) acc *= P.bscale;
        T g0 = cur.g[0][j], g1 = cur.g[1][j], g2 = cur.g[2][j];
        if (!OM1) {
          g0 *= om;
          g1 *= om;
          g2 *= om;
        }
        if (xq >= 1) acc = fma(-g0, xp, acc);
        if (has_y) acc = fma(-g1, sh, acc);
        if (has_in) acc = fma(-g2, ring_in[(s % WV_R) * 32 + lane], acc);
        v = acc;
        if (act) P.xnew[gi0 + xq * dgi] = acc;
      }
      if (act) xp = v;
      if (has_out) ring_out[(s % WV_R) * 32 + lane] = v;
    }
    if (has_out) mb_arrive(&full[wz * NS + st]);
    if (has_in) mb_arrive(&empty[(wz - 1) * NS + st]);
  }
}

// Decomposed ILU(0) pivots (fp64): d_i = a_ii - sum over upstream cells j of
// the same subdomain of a_ij a_ji / d_j.
template <class T, class TC>
__global__ void __launch_bounds__(GT) factor3d_kernel(GP<T, TC> P, const double* A, double* piv, int64_t N) {
  const Sub S = subdomain(P, blockIdx.x);
  const int w = S.len[0], h = S.len[1], d = S.len[2];
  const int lmax = (w - 1) + (h - 1) + (d - 1);
  for (int L = 0; L <= lmax; ++L) {
    for (int q = threadIdx.x; q < h * d; q += GT) {
      const int y = q % h, z = q / h, x = L - y - z;
      if (x < 0 || x >= w) continue;
      const int lc[3] = {x, y, z};
      int64_t gi = 0;
      for (int a = 0; a < 3; ++a) gi += (int64_t)S.gco(a, lc[a]) * P.stride[a];
      double di = A[gi];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        if (lc[a] < 1) continue;
        const int up = S.c[a] ? 1 : 0;
        const int64_t gp = gi + (up ? P.stride[a] : -P.stride[a]);
        // a_ij (entry of i towards j) * a_ji (entry of j towards i) / d_j
        di -= A[(size_t)(1 + ent(a, up)) * N + gi] * A[(size_t)(1 + ent(a, 1 - up)) * N + gp] / __ldcg(piv + gp);
      }
      if (di == 0.0) atomicExch(&P.st->zero_pivot, 1);
      piv[gi] = di;
    }
    __syncthreads();
  }
}

template <class T, class TC, int KIND, bool OM1>
ndiag_status run3d(Handle* h, const GP<T, TC>& P, unsigned nsub, size_t smem, double bytes, bool pencil) {
  static bool attr = false;
  if (!attr) {
    ND_CUDA(cudaFuncSetAttribute(sweep3d_kernel<T, TC, KIND, OM1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 200 * 1024));
    attr = true;
  }
  const int slot = bytes > 0 ? prof_begin(h) : -1;
  ++h->launches;
  if (bytes > 0) ++h->sweep_launches;
  if constexpr (KIND != KIND_SOR) {
    if (pencil && wave_fits(P) && h->w3_wave) {
      const int nw = P.sp[2].len(0);
      const size_t sm = sizeof(T) * (size_t)nw * WvCfg<T>::R * 32 +
                        sizeof(unsigned long long) * 2 * nw * WvCfg<T>::NS;
      static bool wattr = false;
      if (!wattr) {
        ND_CUDA(cudaFuncSetAttribute(sweep3d_wave_kernel<T, TC, KIND, OM1>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        wattr = true;
      }
      sweep3d_wave_kernel<T, TC, KIND, OM1><<<nsub, 32 * nw, sm, h->stream>>>(P);
      ND_CUDA(cudaGetLastError());
      prof_end(h, slot, bytes);
      return NDIAG_OK;
    }
    if (pencil) {
      sweep3d_pencil_kernel<T, TC, KIND, OM1><<<nsub, GT, 2 * sizeof(T) * (size_t)pencil_rows(P), h->stream>>>(P);
      ND_CUDA(cudaGetLastError());
      prof_end(h, slot, bytes);
      return NDIAG_OK;
    }
  }
  // the block passes have at most 3 x (largest side) cells per level: half
  // the threads, so four CTAs fit an SM with up to 128 registers each
  const bool blocks = P.region != REG_ALL && P.region != REG_INTERIOR;
  const int umax = std::max(P.sp[0].len(0), std::max(P.sp[1].len(0), P.sp[2].len(0)));
  // the six-warp layout for the 4-byte passes that solve their blocks themselves (the
  // transposed passes; a forward pass with records runs four warps); the 8-byte
  // variants spill under the six-warp budget
  if (blocks && umax <= 32 && sizeof(T) == 4 && !P.brec) {
    static bool battr = false;
    if (!battr) {
      ND_CUDA(cudaFuncSetAttribute(sweep3d_blocks_kernel<T, TC, KIND, OM1>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
      battr = true;
    }
    sweep3d_blocks_kernel<T, TC, KIND, OM1><<<nsub, 6 * 32, smem, h->stream>>>(P);
  } else {
    sweep3d_kernel<T, TC, KIND, OM1><<<nsub, blocks ? GT / 2 : GT, smem, h->stream>>>(P);
  }
  ND_CUDA(cudaGetLastError());
  prof_end(h, slot, bytes);
  return NDIAG_OK;
}

// rows (h * d) of the largest subdomain
template <class T, class TC>
int pencil_rows(const GP<T, TC>& P) {
  return P.sp[1].len(0) * P.sp[2].len(0);
}
// the wavefront walk: a lane per row along y and a warp per plane along z
template <class T, class TC>
bool wave_fits(const GP<T, TC>& P) {
  return P.sp[1].len(0) <= 32 && P.sp[2].len(0) <= 32;
}

// Level-ordered copy of a scaled set (7 arrays) in the frame of P (the
// reference frame): one thread per cell.
template <class T, class TC>
__global__ void level_layout_kernel(GP<T, TC> P, const TC* src, TC* dst, int64_t N) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const int gx = (int)(i % P.n[0]);
    const int64_t rest = i / P.n[0];
    const int gy = (int)(rest % P.n[1]), gz = (int)(rest / P.n[1]);
    const int ix = split_find(P.sp[0], gx), iy = split_find(P.sp[1], gy), iz = split_find(P.sp[2], gz);
    const unsigned b = (unsigned)(ix + P.sp[0].p * (iy + P.sp[1].p * iz));
    const Sub S = subdomain(P, b);
    int l[3];
    const int g[3] = {gx, gy, gz};
    for (int a = 0; a < 3; ++a) l[a] = S.c[a] ? S.g0[a] + S.len[a] - 1 - g[a] : g[a] - S.g0[a];
    const int64_t o = (int64_t)b * P.lev_sub + (int64_t)(l[0] + l[1] + l[2]) * P.lev_hd0 + l[1] + P.lev_h0 * l[2];
    for (int k = 0; k < 7; ++k) dst[k * P.lev_arr + o] = src[(int64_t)k * N + i];
  }
}

// The level-ordered copy of `set` in the frame of the forward phase, built
// when missing or stale; fills the lev fields of P (null when not applicable).
template <class T, class TC>
ndiag_status attach_levels(Handle* h, ScaledSet& set, GP<T, TC>& P, int mode) {
  P.lev = nullptr;
  if (mode != NDIAG_DECOMPOSED || h->dim != 3) return NDIAG_OK;
  GP<T, TC> R = P;  // reference frame: the forward phase
  R.base = base_corner(3, fwd_phase(3));
  const int w0 = P.sp[0].len(0), h0 = P.sp[1].len(0), d0 = P.sp[2].len(0);
  R.lev_h0 = h0;
  R.lev_hd0 = h0 * d0;
  R.lev_sub = (int64_t)(w0 + h0 + d0 - 2) * R.lev_hd0;
  const int64_t nsub = (int64_t)P.sp[0].p * P.sp[1].p * P.sp[2].p;
  R.lev_arr = nsub * R.lev_sub;
  const size_t bytes = sizeof(TC) * 7 * (size_t)R.lev_arr;
  if (!set.lev || set.lev_bytes != bytes) {
    dev_free(set.lev, set.lev_bytes, h->stream);
    set.lev = dev_alloc(bytes, h->stream);
    set.lev_bytes = set.lev ? bytes : 0;
    set.lev_version = ~0u;
    if (!set.lev) return NDIAG_OK;  // no room: the natural arrays serve
  }
  if (set.lev_version != set.version) {
    ++h->launches;
    level_layout_kernel<T, TC><<<h->sm_count * 8, 256, 0, h->stream>>>(R, (const TC*)set.base, (TC*)set.lev, h->N);
    ND_CUDA(cudaGetLastError());
    set.lev_version = set.version;
  }
  P.lev = (const TC*)set.lev;
  P.lev_arr = R.lev_arr;
  P.lev_sub = R.lev_sub;
  P.lev_h0 = R.lev_h0;
  P.lev_hd0 = R.lev_hd0;
  P.lev_flip = P.base ^ R.base;
  return NDIAG_OK;
}

// The forward block records of (set, phase, kind, partition), built on first
// use and rebuilt when the set's values change; P.brec stays null when there
// is no room (the block solves then gather their operands themselves).
template <class T, class TC>
ndiag_status attach_records(Handle* h, const ScaledSet& set, GP<T, TC>& P, int kind) {
  P.brec = nullptr;
  const bool tr = P.transposed != 0;
  const int key = kind + (tr ? 16 : 0);
  const int64_t nsub = (int64_t)P.sp[0].p * P.sp[1].p * P.sp[2].p;
  const int64_t total = nsub * P.twin_slots;
  const size_t bytes = sizeof(BRec<T>) * (size_t)total;
  const int s0 = P.sp[0].p, s1 = P.sp[1].p * 65536 + P.sp[2].p;
  PackCache* pc = nullptr;
  for (PackCache& c : h->brec3d)
    if (c.t == P.base && c.kind == key && c.sub0 == s0 && c.sub1 == s1) pc = &c;
  if (!pc) {
    h->brec3d.push_back(PackCache{});
    pc = &h->brec3d.back();
    pc->t = P.base;
    pc->kind = key;
    pc->sub0 = s0;
    pc->sub1 = s1;
  }
  if (!pc->buf || pc->bytes != bytes || pc->set_base != set.base || pc->set_version != set.version) {
    if (pc->bytes != bytes) {
      dev_free(pc->buf, pc->bytes, h->stream);
      pc->buf = (double*)dev_alloc(bytes, h->stream);
      pc->bytes = pc->buf ? bytes : 0;
    }
    if (!pc->buf) {
      pc->set_base = nullptr;
      return NDIAG_OK;
    }
    const unsigned grid = (unsigned)std::min<int64_t>((total + 127) / 128, (int64_t)h->sm_count * 16);
    ++h->launches;
    if (tr)
      block_record_kernel<T, TC, KIND_TRI_UNIT, true><<<grid, 128, 0, h->stream>>>(P, (BRec<T>*)pc->buf, total);
    else if (kind == KIND_TRI_SCALED)
      block_record_kernel<T, TC, KIND_TRI_SCALED, false><<<grid, 128, 0, h->stream>>>(P, (BRec<T>*)pc->buf, total);
    else
      block_record_kernel<T, TC, KIND_TRI_UNIT, false><<<grid, 128, 0, h->stream>>>(P, (BRec<T>*)pc->buf, total);
    ND_CUDA(cudaGetLastError());
    pc->set_base = set.base;
    pc->set_version = set.version;
  }
  P.brec = pc->buf;
  return NDIAG_OK;
}

template <class T, class TC>
GP<T, TC> params(Handle* h, int mode, int64_t t, const ScaledSet& set, const void* rhs, const void* xold,
                 void* xnew, size_t& smem, unsigned& nsub) {
  GP<T, TC> P{};
  const bool nat = mode == NDIAG_NATURAL || mode == MODE_NATURAL_REV;
  P.dim = h->dim;
  for (int a = 0; a < 3; ++a) {
    P.n[a] = (int)h->n[a];
    const int p = nat ? 1 : h->sub[a];
    P.sp[a] = Split{p, P.n[a] / p, P.n[a] % p};
  }
  P.stride[0] = 1;
  P.stride[1] = P.n[0];
  P.stride[2] = (int64_t)P.n[0] * P.n[1];
  P.base = nat ? (mode == MODE_NATURAL_REV ? (1 << h->dim) - 1 : 0) : base_corner(h->dim, t);
  P.coupled = nat ? 0 : 1;
  const size_t N = (size_t)h->N;
  const TC* b = (const TC*)set.base;
  P.inv = b;
  for (int e = 0; e < 6; ++e) P.c[e] = b + (size_t)(1 + e) * N;
  P.rhs = (const T*)rhs;
  P.xold = (const T*)xold;
  P.xnew = (T*)xnew;
  P.st = h->status;
  const int w = P.sp[0].len(0), hh = P.sp[1].len(0), d = P.sp[2].len(0);
  P.twin_slots = P.coupled ? twin_store_size(w, hh, d) : 0;
  smem = sizeof(T) * (size_t)P.twin_slots;
  nsub = (unsigned)(P.sp[0].p * P.sp[1].p * P.sp[2].p);
  return P;
}

template <class T, class TC>
ndiag_status sweep3d_t(Handle* h, int kind, int mode, int64_t t, const double* omega, const ScaledSet& set,
                       const void* rhs, const void* xold, void* xnew, double beta_scale, bool transposed) {
  size_t smem = 0;
  unsigned nsub = 0;
  GP<T, TC> P = params<T, TC>(h, mode, t, set, rhs, xold, xnew, smem, nsub);
  if (smem > 200 * 1024) {
    set_error("3D subdomains too large for the twin store");
    return NDIAG_EINVAL;
  }
  bool om1 = beta_scale == 1.0;
  for (int k = 0; k < 8; ++k) {
    const double wv = omega ? (mode == NDIAG_DECOMPOSED ? omega[k] : omega[0]) : 1.0;
    P.om[k] = (T)wv;
    if (wv != 1.0) om1 = false;
  }
  P.bscale = (T)beta_scale;
  const double cellbytes = kind == KIND_SOR ? 9.0 * sizeof(TC) + 3.0 * sizeof(T)
                                            : (kind == KIND_TRI_SCALED ? 4.0 : 3.0) * sizeof(TC) + 2.0 * sizeof(T);
  const double bytes = cellbytes * (double)h->N;
  // the pencil walk: triangular kinds, rows of the largest subdomain within KR per thread
  const bool pencil = kind != KIND_SOR && pencil_rows(P) <= KR * GT;
  if (pencil) ND_TRY(attach_levels(h, const_cast<ScaledSet&>(set), P, mode));  // lev is a cache of set
  // one sweep's bytes go with its last (forward) or first (transposed) launch
  double b_now = bytes;
  auto go = [&](auto kt, auto o1) -> ndiag_status {
    constexpr int K = decltype(kt)::value;
    constexpr bool O = decltype(o1)::value;
    const bool pen = pencil && P.region == REG_INTERIOR;
    const ndiag_status st = run3d<T, TC, K, O>(h, P, nsub, smem, b_now, pen);
    return st;
  };
  using S0 = std::integral_constant<int, KIND_SOR>;
  using S1 = std::integral_constant<int, KIND_TRI_SCALED>;
  using S2 = std::integral_constant<int, KIND_TRI_UNIT>;
  using BT = std::true_type;
  using BF = std::false_type;
  if (!transposed) {
    P.region = REG_ALL;
    if (kind == KIND_SOR) return om1 ? go(S0(), BT()) : go(S0(), BF());
    auto fwd = [&](auto kt) -> ndiag_status {
      if (!pencil) {
        P.region = REG_ALL;
        return om1 ? go(kt, BT()) : go(kt, BF());
      }
      if (P.coupled) {  // the coupled blocks first, then the one-cell blocks
        P.region = REG_BLOCKS;
        b_now = 0.0;
        if (om1 && h->w3_wave) ND_TRY(attach_records(h, set, P, decltype(kt)::value));
        ND_TRY(om1 ? go(kt, BT()) : go(kt, BF()));
        P.brec = nullptr;
      }
      P.region = REG_INTERIOR;
      b_now = bytes;
      return om1 ? go(kt, BT()) : go(kt, BF());
    };
    if (kind == KIND_TRI_SCALED) return fwd(S1());
    return fwd(S2());
  }
  // (D + w L^T) y = v: interiors, then faces, edges, corners (earlier passes
  // read from global memory); only the interior pass counts the bytes
  P.transposed = 1;
  const int last = P.coupled ? (h->dim == 3 ? REG_CORNERS : REG_EDGES) : REG_INTERIOR;
  for (int r = REG_INTERIOR; r <= last; ++r) {
    P.region = r;
    b_now = r == REG_INTERIOR ? bytes : 0.0;
    // the face and edge passes solve recorded blocks (one record set for both)
    if (r == REG_FACES && om1 && h->w3_wave && h->dim == 3) ND_TRY(attach_records(h, set, P, KIND_TRI_UNIT));
    ND_TRY(om1 ? go(S2(), BT()) : go(S2(), BF()));
  }
  P.brec = nullptr;
  return NDIAG_OK;
}

}  // namespace

// kinds KIND_SOR / KIND_TRI_SCALED / KIND_TRI_UNIT; `transposed` solves with
// the transposed set (D + w L^T) in the phase's frame
ndiag_status launch_sweep3d(Handle* h, int kind, int mode, int64_t t, const double* omega, const ScaledSet& set,
                            const void* rhs, const void* xold, void* xnew, double beta_scale, bool transposed) {
  switch (h->precision) {
    case NDIAG_FP64:
      return sweep3d_t<double, double>(h, kind, mode, t, omega, set, rhs, xold, xnew, beta_scale, transposed);
    case NDIAG_FP32:
      return sweep3d_t<float, float>(h, kind, mode, t, omega, set, rhs, xold, xnew, beta_scale, transposed);
    default:
      return sweep3d_t<float, __half>(h, kind, mode, t, omega, set, rhs, xold, xnew, beta_scale, transposed);
  }
}

ndiag_status launch_ilu_factor3d_into(Handle* h, int mode, double* out) {
  size_t smem = 0;
  unsigned nsub = 0;
  GP<double, double> P = params<double, double>(h, mode, fwd_phase(h->dim), h->sor, nullptr, nullptr, nullptr,
                                                smem, nsub);
  ++h->launches;
  factor3d_kernel<double, double><<<nsub, GT, 0, h->stream>>>(P, h->A64, out, h->N);
  ND_CUDA(cudaGetLastError());
  return NDIAG_OK;
}

}  // namespace nd
