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
#include "sweep_common.cuh"

namespace nd {
namespace {

using namespace sweep;

constexpr int GT = 256;  // threads per CTA

enum { REG_ALL = 0, REG_INTERIOR = 1, REG_FACES = 2, REG_EDGES = 3, REG_CORNERS = 4 };

template <class T, class TC>
struct GP {
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
};

struct Sub {
  int idx[3], g0[3], len[3], c[3], t[3];
  __device__ int gco(int a, int l) const { return c[a] ? g0[a] + len[a] - 1 - l : g0[a] + l; }
};

// entry index (0-based in c[]) of the neighbour along axis a towards -a / +a
__device__ __forceinline__ int ent(int a, int plus) { return 2 * a + plus; }

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
    default: return true;
  }
}

template <class T, class TC, int KIND, bool OM1>
__global__ void __launch_bounds__(GT) sweep3d_kernel(GP<T, TC> P) {
  extern __shared__ __align__(16) unsigned char gsm[];
  T* tw = reinterpret_cast<T*>(gsm);
  const Sub S = subdomain(P, blockIdx.x);
  const int w = S.len[0], h = S.len[1], d = S.len[2];
  const TwinIdx TI = twin_index(w, h, d);
  const int lmax = (w - 1) + (h - 1) + (d - 1);
  const int tcode = S.t[0] | (S.t[1] << 1) | (S.t[2] << 2);
  for (int it = 0; it <= lmax; ++it) {
    const int L = P.transposed ? lmax - it : it;
    for (int q = threadIdx.x; q < h * d; q += GT) {
      const int y = q % h, z = q / h, x = L - y - z;
      if (x < 0 || x >= w) continue;
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
            for (int a = 0; a < P.dim; ++a) {
              const int dn = S.c[a] ? 0 : 1;
              const int gd = gc[a] + (dn ? 1 : -1);
              if (gd >= 0 && gd < P.n[a])
                e = fma(-ldco<T, TC>(P.c[ent(a, dn)] + gi), __ldg(P.xold + gi + (dn ? P.stride[a] : -P.stride[a])), e);
              const int gu = gc[a] + (dn ? -1 : 1);
              if (own[a] == 0 && gu >= 0 && gu < P.n[a])
                e = fma(-ldco<T, TC>(P.c[ent(a, 1 - dn)] + gi), __ldg(P.xold + gi + (dn ? -P.stride[a] : P.stride[a])), e);
            }
            acc = OM1 ? e : fma(om, e, (T(1) - om) * __ldg(P.xold + gi));
          } else if (KIND == KIND_TRI_SCALED) {
            acc = ldco<T, TC>(P.inv + gi) * __ldg(P.rhs + gi);
            if (!OM1) acc *= P.bscale;
          } else {
            acc = __ldg(P.rhs + gi);
          }
          for (int a = 0; a < P.dim; ++a) {
            if (own[a] < 1) continue;
            const int up = S.c[a] ? 1 : 0;
            T g = ldco<T, TC>(P.c[ent(a, up)] + gi);
            if (!OM1) g *= om;
            acc = fma(-g, __ldcg(P.xnew + gi + (up ? P.stride[a] : -P.stride[a])), acc);
          }
        } else {
          acc = __ldg(P.rhs + gi);
          for (int a = 0; a < P.dim; ++a) {
            if (own[a] + 1 >= S.len[a]) continue;
            const int dn = S.c[a] ? 0 : 1;
            T g = ldco<T, TC>(P.c[ent(a, dn)] + gi);
            if (!OM1) g *= om;
            acc = fma(-g, __ldcg(P.xnew + gi + (dn ? P.stride[a] : -P.stride[a])), acc);
          }
        }
        P.xnew[gi] = acc;
        continue;
      }
      // canonical member order: bit r of a member index <-> r-th coupled axis,
      // set when the member has the larger global coordinate along it
      int axes[3], nC = 0;
      for (int a = 0; a < 3; ++a)
        if (C >> a & 1) axes[nC++] = a;
      const int n = 1 << nC;
      int mo = 0;  // own member
      for (int r = 0; r < nC; ++r)
        if (S.c[axes[r]] == 0) mo |= 1 << r;
      T M[8][8], hv[8];
      int64_t gidx[8];
      for (int m = 0; m < n; ++m) {
        int lc[3] = {own[0], own[1], own[2]}, sub = 0;
        for (int r = 0; r < nC; ++r)
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
        for (int k = 0; k < n; ++k) M[m][k] = T(0);
        M[m][m] = T(1);
        T acc;
        if (!P.transposed) {
          if (KIND == KIND_SOR) {
            T e = ldco<T, TC>(P.inv + gi) * __ldg(P.rhs + gi);
            for (int a = 0; a < P.dim; ++a) {
              const int dn = cm[a] ? 0 : 1;  // downstream side of the member along a
              const int gd = gc[a] + (dn ? 1 : -1);
              if (gd >= 0 && gd < P.n[a])
                e = fma(-ldco<T, TC>(P.c[ent(a, dn)] + gi), __ldg(P.xold + gi + (dn ? P.stride[a] : -P.stride[a])), e);
              const bool implicit_up = (C >> a & 1) || lc[a] >= 1;
              const int gu = gc[a] + (dn ? -1 : 1);
              if (!implicit_up && gu >= 0 && gu < P.n[a])
                e = fma(-ldco<T, TC>(P.c[ent(a, 1 - dn)] + gi), __ldg(P.xold + gi + (dn ? -P.stride[a] : P.stride[a])), e);
            }
            acc = OM1 ? e : fma(om, e, (T(1) - om) * __ldg(P.xold + gi));
          } else if (KIND == KIND_TRI_SCALED) {
            acc = ldco<T, TC>(P.inv + gi) * __ldg(P.rhs + gi);
            if (!OM1) acc *= P.bscale;
          } else {
            acc = __ldg(P.rhs + gi);
          }
          // upstream neighbours: block partners, or earlier blocks' members
          for (int a = 0; a < P.dim; ++a) {
            const int up = cm[a] ? 1 : 0;  // upstream side of the member along a
            if (C >> a & 1) {
              int r = 0;
              while (axes[r] != a) ++r;
              T g = ldco<T, TC>(P.c[ent(a, up)] + gi);
              if (!OM1) g *= om;
              M[m][m ^ (1 << r)] = g;
            } else if (lc[a] >= 1) {
              T g = ldco<T, TC>(P.c[ent(a, up)] + gi);
              if (!OM1) g *= om;
              const int64_t gp = gi + (up ? P.stride[a] : -P.stride[a]);
              T v;
              if (sub == 0) {
                v = __ldcg(P.xnew + gp);
              } else {
                int pc[3] = {lc[0], lc[1], lc[2]};
                pc[a] -= 1;
                v = tw[TI.slot(sub, pc)];
              }
              acc = fma(-g, v, acc);
            }
          }
        } else {
          // transposed: dependents are the downstream neighbours inside the
          // member's own subdomain, and the block partners
          acc = __ldg(P.rhs + gi);
          for (int a = 0; a < P.dim; ++a) {
            const int up = cm[a] ? 1 : 0, dn = 1 - up;
            if (C >> a & 1) {
              int r = 0;
              while (axes[r] != a) ++r;
              T g = ldco<T, TC>(P.c[ent(a, up)] + gi);
              if (!OM1) g *= om;
              M[m][m ^ (1 << r)] = g;
            }
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
            if (!inside) continue;
            T g = ldco<T, TC>(P.c[ent(a, dn)] + gi);
            if (!OM1) g *= om;
            const int64_t gq = gi + (dn ? P.stride[a] : -P.stride[a]);
            T v;
            if (sub == 0 || twin_axis) {
              v = __ldcg(P.xnew + gq);
            } else {
              // same twin subset one step downstream: this launch's store
              // if that block is of the same kind, else an earlier launch
              int pc[3] = {lc[0], lc[1], lc[2]};
              pc[a] += 1;
              int oc[3] = {own[0], own[1], own[2]};
              oc[a] += 1;
              const int C2 = ((oc[0] == 0) | ((oc[1] == 0) << 1) | ((oc[2] == 0) << 2)) & tcode;
              v = (__popc(C2) == nC) ? tw[TI.slot(sub, pc)] : __ldcg(P.xnew + gq);
            }
            acc = fma(-g, v, acc);
          }
        }
        hv[m] = acc;
      }
      // (I + G) x = h, elimination in canonical order (diagonally dominant: no pivoting)
      for (int k = 0; k < n; ++k) {
        const T piv = M[k][k];
        for (int i = k + 1; i < n; ++i) {
          const T f = M[i][k] / piv;
          if (f != T(0)) {
            for (int j = k + 1; j < n; ++j) M[i][j] = fma(-f, M[k][j], M[i][j]);
            hv[i] = fma(-f, hv[k], hv[i]);
          }
        }
      }
      T xs[8];
      for (int k = n - 1; k >= 0; --k) {
        T s = hv[k];
        for (int j = k + 1; j < n; ++j) s = fma(-M[k][j], xs[j], s);
        xs[k] = s / M[k][k];
      }
      for (int m = 0; m < n; ++m) {
        if (m == mo) {
          P.xnew[gidx[m]] = xs[m];
        } else {
          int lc[3] = {own[0], own[1], own[2]}, sub = 0;
          for (int r = 0; r < nC; ++r)
            if (((m ^ mo) >> r) & 1) {
              lc[axes[r]] = -1;
              sub |= 1 << axes[r];
            }
          tw[TI.slot(sub, lc)] = xs[m];
        }
      }
    }
    __syncthreads();
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
      for (int a = 0; a < P.dim; ++a) {
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
ndiag_status run3d(Handle* h, const GP<T, TC>& P, unsigned nsub, size_t smem, double bytes) {
  static bool attr = false;
  if (!attr) {
    ND_CUDA(cudaFuncSetAttribute(sweep3d_kernel<T, TC, KIND, OM1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 200 * 1024));
    attr = true;
  }
  const int slot = prof_begin(h);
  ++h->launches;
  ++h->sweep_launches;
  sweep3d_kernel<T, TC, KIND, OM1><<<nsub, GT, smem, h->stream>>>(P);
  ND_CUDA(cudaGetLastError());
  prof_end(h, slot, bytes);
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
  smem = P.coupled ? sizeof(T) * (size_t)twin_store_size(w, hh, d) : 0;
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
  auto go = [&](auto kt, auto o1) -> ndiag_status {
    constexpr int K = decltype(kt)::value;
    constexpr bool O = decltype(o1)::value;
    return run3d<T, TC, K, O>(h, P, nsub, smem, bytes);
  };
  using S0 = std::integral_constant<int, KIND_SOR>;
  using S1 = std::integral_constant<int, KIND_TRI_SCALED>;
  using S2 = std::integral_constant<int, KIND_TRI_UNIT>;
  using BT = std::true_type;
  using BF = std::false_type;
  if (!transposed) {
    P.region = REG_ALL;
    if (kind == KIND_SOR) return om1 ? go(S0(), BT()) : go(S0(), BF());
    if (kind == KIND_TRI_SCALED) return om1 ? go(S1(), BT()) : go(S1(), BF());
    return om1 ? go(S2(), BT()) : go(S2(), BF());
  }
  // (D + w L^T) y = v: interiors, then faces, edges, corners (earlier passes
  // read from global memory); only the interior pass counts the bytes
  P.transposed = 1;
  const int last = P.coupled ? (h->dim == 3 ? REG_CORNERS : REG_EDGES) : REG_INTERIOR;
  for (int r = REG_INTERIOR; r <= last; ++r) {
    P.region = r;
    ND_TRY(om1 ? go(S2(), BT()) : go(S2(), BF()));
  }
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
