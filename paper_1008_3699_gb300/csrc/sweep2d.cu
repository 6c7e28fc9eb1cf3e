// Decomposed sequential sweep on 2D 5-point structured matrices (sm_103a).
//
// One sweep of phase t solves, row by row in the order of the paper's
// multi-frontal sweep,  (Delta + L_J) x = g  (Eqs. sor2d_sw..sor2d_nw; coupled
// start nodes by Eqs. 2d:sor4b4 and 2d:sor2b2; splitting form Eq. ca2d:matiter),
// written per cell with scaled coefficients as
//        x_i = beta_i - sum_{j in J_i} gamma_ij x_j .
//
// GPU layout. Each subdomain is an independent tile. Its cells are visited in a
// local frame reflected so that the sweep always runs from local (0,0) towards
// +x,+y. A subdomain whose start side along an axis is an interface shares that
// interface with a neighbour that also starts there (the schedule flips the
// direction bit between neighbours), so the two start lines form coupled pairs
// (Eq. 2d:sor2b2) and the four start corners form a 4x4 system
// (Eq. 2d:sor4b4). Instead of synchronising with the neighbour, a CTA
// recomputes the neighbour's start line ("twin" line at local -1) from old
// values two cells deep -- the paper's halo of two rows/columns (Sec. 3,
// "Data structure") -- and solves each pair itself. Both CTAs evaluate every
// coupled value with the same operation sequence, so the twin and the owner
// agree bit for bit.
//
// Inside a tile a warp owns a band of 32 rows (lane = row) and walks the
// columns as a skewed anti-diagonal wavefront (lane l handles column s - l at
// step s); the south value arrives from lane l-1 by a register shuffle. A CTA
// holds NW consecutive bands ("slab"); band b+1 receives band b's top row
// through a shared-memory ring, published in chunks of CH columns. A subdomain
// taller than one slab (the natural ordering is one subdomain) is split into
// slabs taken in ticket order by CTAs; slab j+1 reads slab j's top row from
// global memory behind a release/acquire progress flag. Every wait is bounded:
// on timeout the warp records NDIAG_ETIMEOUT in the status word and returns.
#include "internal.h"

namespace nd {
namespace {

constexpr int NW = 4;         // bands (warps) per CTA
constexpr int BH = 32;        // rows per band
constexpr int CH = 16;        // handoff chunk (columns)
constexpr int RING = 64;      // shared-memory ring per band boundary (columns)
constexpr long long WAIT_CYCLES = 4000000000LL;  // ~2 s at 2 GHz
constexpr unsigned FULL = 0xffffffffu;

enum { KIND_FACTOR = 100 };

template <class T, class TC>
struct SweepP {
  int nx, ny;
  Split sx, sy;
  int base;        // start corner of subdomain (0,0)
  int spp;         // slabs per subdomain
  int use_ticket;  // slabs taken in ticket order (multi-slab subdomains)
  int coupled;     // 0: no interface coupling (natural ordering, reverse pass)
  int rev;         // reverse interior pass of the SSOR transposed solve
  const TC* inv;   // 1 / pivot
  const TC* c[4];  // scaled off-diagonals, entries W E S N
  const T* rhs;
  const T* xold;
  T* xnew;
  const double* A;  // raw fp64 matrix (factor kernel)
  T om[4];          // relaxation per start corner
  T bscale;         // factor on beta (KIND_TRI_SCALED)
  unsigned* ticket;
  unsigned* flags;  // per slab: columns of the top row published
  T* twin_hand;     // per slab: twin value of the top row
  DevStatus* st;
};

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

// Bounded wait until *p >= v (warp-uniform). Returns false on timeout.
__device__ bool wait_smem(const volatile int* p, int v, DevStatus* st) {
  if (*p >= v) return true;
  const long long t0 = clock64();
  while (*p < v) {
    if (clock64() - t0 > WAIT_CYCLES) {
      atomicExch(&st->timeout, 1);
      return false;
    }
    __nanosleep(32);
  }
  __threadfence_block();
  return true;
}
__device__ bool wait_gmem(const unsigned* p, unsigned v, DevStatus* st) {
  if (ld_acquire(p) >= v) return true;
  const long long t0 = clock64();
  while (ld_acquire(p) < v) {
    if (clock64() - t0 > WAIT_CYCLES) {
      atomicExch(&st->timeout, 1);
      return false;
    }
    __nanosleep(64);
  }
  return true;
}

// beta and the two implicit coefficients of one cell. jx / jy are the entries
// (0 W, 1 E, 2 S, 3 N) of the cell's implicit x / y neighbour; the opposite
// entries hold old values (SOR only). The x term is always taken before the y
// term so that the owner of a cell and a CTA recomputing it as a twin perform
// the same operations.
template <class T, class TC, int KIND>
__device__ __forceinline__ void cell_bg(const SweepP<T, TC>& P, int gx, int gy, int jx, int jy,
                                        T om, T& beta, T& gjx, T& gjy) {
  const int64_t gi = (int64_t)gy * P.nx + gx;
  gjx = om * ldco<T, TC>(P.c[jx] + gi);
  gjy = om * ldco<T, TC>(P.c[jy] + gi);
  if (KIND == KIND_SOR) {
    T acc = ldco<T, TC>(P.inv + gi) * __ldg(P.rhs + gi);
    const int ox = jx ^ 1, oy = jy ^ 1;
    const int xo = gx + (ox == 1 ? 1 : -1);
    if (xo >= 0 && xo < P.nx) acc = fma(-ldco<T, TC>(P.c[ox] + gi), __ldg(P.xold + gi + (xo - gx)), acc);
    const int yo = gy + (oy == 3 ? 1 : -1);
    if (yo >= 0 && yo < P.ny)
      acc = fma(-ldco<T, TC>(P.c[oy] + gi), __ldg(P.xold + gi + (int64_t)(yo - gy) * P.nx), acc);
    beta = fma(om, acc, (T(1) - om) * __ldg(P.xold + gi));
  } else if (KIND == KIND_TRI_SCALED) {
    beta = P.bscale * ldco<T, TC>(P.inv + gi) * __ldg(P.rhs + gi);
  } else {
    beta = __ldg(P.rhs + gi);
  }
}

// Coupled pair x_a = h_a - g_ab x_b, x_b = h_b - g_ba x_a. The formula is
// symmetric in (a, b), so both CTAs that solve a pair get identical bits.
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
  // eliminate slots 1 and 2, solve the 2x2 in slots 0 and 3
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

template <class T, class TC, int KIND>
__global__ void __launch_bounds__(NW * 32) sweep2d_kernel(SweepP<T, TC> P) {
  __shared__ T ring[NW][RING];
  __shared__ T ring_tw[NW];
  __shared__ int prod[NW];
  __shared__ int cons[NW];
  __shared__ unsigned s_ticket;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x < NW) {
    prod[threadIdx.x] = 0;
    cons[threadIdx.x] = 0;
  }
  if (P.use_ticket && threadIdx.x == 0) s_ticket = atomicAdd(P.ticket, 1u);
  __syncthreads();
  const unsigned slab_id = P.use_ticket ? s_ticket : blockIdx.x;

  const unsigned sub = slab_id / P.spp, j = slab_id % P.spp;
  const int ix = (int)(sub % (unsigned)P.sx.p), iy = (int)(sub / (unsigned)P.sx.p);
  if (iy >= P.sy.p) return;
  const int gx0 = P.sx.lo(ix), w = P.sx.len(ix), gy0 = P.sy.lo(iy), h = P.sy.len(iy);
  const int c = P.base ^ (ix & 1) ^ ((iy & 1) << 1);
  const int cx = c & 1, cy = (c >> 1) & 1;
  const bool tx = KIND != KIND_FACTOR && P.coupled && (cx ? (gx0 + w < P.nx) : (gx0 > 0));
  const bool ty = KIND != KIND_FACTOR && P.coupled && (cy ? (gy0 + h < P.ny) : (gy0 > 0));
  const int bands = (h + BH - 1) / BH;
  const int band = (int)j * NW + warp;
  if (band >= bands) return;
  // reverse pass: the last column / row border coupled interfaces of the
  // forward phase and are solved afterwards by the edge kernel
  const bool skip_x = P.rev && (cx ? (gx0 > 0) : (gx0 + w < P.nx));
  const bool skip_y = P.rev && (cy ? (gy0 > 0) : (gy0 + h < P.ny));

  const int lW = cx ? 1 : 0, lE = lW ^ 1, lS = cy ? 3 : 2, lN = lS ^ 1;
  auto gxl = [&](int lx) { return cx ? gx0 + w - 1 - lx : gx0 + lx; };
  auto gyl = [&](int ly) { return cy ? gy0 + h - 1 - ly : gy0 + ly; };
  const T om_p = P.om[c], om_q = P.om[c ^ 2], om_r = P.om[c ^ 1], om_s = P.om[c ^ 3];

  const int ly = band * BH + lane;
  const bool row_on = ly < h;
  const int gy = gyl(row_on ? ly : 0);
  const bool has_cons = band + 1 < bands;
  const bool smem_prod = has_cons && warp < NW - 1;
  const bool gmem_prod = has_cons && warp == NW - 1;
  const bool smem_cons = band > 0 && warp > 0;
  const bool gmem_cons = band > 0 && warp == 0;
  const unsigned slab_g = sub * P.spp + j;

  T x_prev = T(0), tw = T(0), q_prev = T(0), hs = T(0), tw_in = T(0);
  const int steps = w + BH - 1;
  for (int s = 0; s < steps; ++s) {
    // ---- receive the band below's top row, CH columns at a time
    if ((smem_cons || gmem_cons) && (s % CH) == 0 && s < w) {
      const int need = min(s + CH, w);
      bool ok;
      if (smem_cons) ok = wait_smem(&prod[warp - 1], need, P.st);
      else ok = wait_gmem(&P.flags[slab_g - 1], (unsigned)need, P.st);
      if (!ok) return;
      if (lane < CH && s + lane < w) {
        if (smem_cons) hs = ring[warp - 1][(s + lane) % RING];
        else hs = __ldcg(P.xnew + (int64_t)gyl(band * BH - 1) * P.nx + gxl(s + lane));
      }
      if (s == 0 && lane == 0) tw_in = smem_cons ? ring_tw[warp - 1] : __ldcg(P.twin_hand + slab_g - 1);
      __syncwarp();
      if (smem_cons && lane == 0) ((volatile int*)cons)[warp - 1] = need;
    }
    // ---- producer back-pressure on the shared ring (lane 31 writes column s-31)
    if (smem_prod) {
      const int lx31 = s - (BH - 1);
      if (lx31 >= 0 && lx31 < w && (lx31 % CH) == 0 && lx31 + CH > RING) {
        if (!wait_smem(&cons[warp], lx31 + CH - RING, P.st)) return;
      }
    }

    const T xS_sh = __shfl_up_sync(FULL, x_prev, 1);
    const T tw_sh = __shfl_up_sync(FULL, tw, 1);
    const T hS = __shfl_sync(FULL, hs, s % CH);
    const int lx = s - lane;
    if (row_on && lx >= 0 && lx < w && !((skip_x && lx == w - 1) || (skip_y && ly == h - 1))) {
      const int gx = gxl(lx);
      const int64_t gi = (int64_t)gy * P.nx + gx;
      const T xS = lane > 0 ? xS_sh : (band == 0 ? T(0) : hS);
      T x;
      if (KIND == KIND_FACTOR) {
        // d~_i = a_ii - sum over upstream neighbours in the subdomain of
        // a_ij a_ji / d~_j (mutual interface pairs excluded: none here).
        double acc = P.A[gi];
        if (lx > 0) {
          const int64_t gj = gi + (lW == 1 ? 1 : -1);
          acc -= P.A[(int64_t)(1 + lW) * (P.nx * (int64_t)P.ny) + gi] *
                 P.A[(int64_t)(1 + lE) * (P.nx * (int64_t)P.ny) + gj] / (double)x_prev;
        }
        if (ly > 0) {
          const int64_t gj = gi + (lS == 3 ? P.nx : -P.nx);
          acc -= P.A[(int64_t)(1 + lS) * (P.nx * (int64_t)P.ny) + gi] *
                 P.A[(int64_t)(1 + lN) * (P.nx * (int64_t)P.ny) + gj] / (double)xS;
        }
        if (acc == 0.0) atomicExch(&P.st->zero_pivot, 1);
        x = (T)acc;
      } else {
        T beta, gW, gS;
        cell_bg<T, TC, KIND>(P, gx, gy, lW, lS, om_p, beta, gW, gS);
        if (lx == 0 && tx) {
          // own start column pairs with the twin column of the x-neighbour
          T br, grE, grS;
          cell_bg<T, TC, KIND>(P, gxl(-1), gy, lE, lS, om_r, br, grE, grS);
          if (ly == 0 && ty) {
            T bq, gqW, gqN, bs, gsE, gsN;
            cell_bg<T, TC, KIND>(P, gx, gyl(-1), lW, lN, om_q, bq, gqW, gqN);
            cell_bg<T, TC, KIND>(P, gxl(-1), gyl(-1), lE, lN, om_s, bs, gsE, gsN);
            // canonical slots by global position
            const int sp = (1 ^ cx) | ((1 ^ cy) << 1);  // local (0,0)
            const int sq = (1 ^ cx) | (cy << 1);        // local (0,-1)
            const int sr = cx | ((1 ^ cy) << 1);        // local (-1,0)
            const int ss = cx | (cy << 1);              // local (-1,-1)
            T hh[4], gx4[4], gy4[4], xx[4];
            hh[sp] = beta; gx4[sp] = gW;  gy4[sp] = gS;
            hh[sq] = bq;   gx4[sq] = gqW; gy4[sq] = gqN;
            hh[sr] = br;   gx4[sr] = grE; gy4[sr] = grS;
            hh[ss] = bs;   gx4[ss] = gsE; gy4[ss] = gsN;
            corner_solve(hh, gx4, gy4, xx);
            x = xx[sp];
            tw = xx[sr];
            q_prev = xx[sq];
          } else {
            const T rS = lane > 0 ? tw_sh : (band == 0 ? T(0) : tw_in);
            pair_solve(fma(-gS, xS, beta), gW, fma(-grS, rS, br), grE, x, tw);
          }
        } else if (ly == 0 && ty) {
          // own start row pairs with the twin row of the y-neighbour
          T bq, gqW, gqN;
          cell_bg<T, TC, KIND>(P, gx, gyl(-1), lW, lN, om_q, bq, gqW, gqN);
          const T xW = lx == 0 ? T(0) : x_prev;
          const T qW = lx == 0 ? T(0) : q_prev;
          pair_solve(fma(-gW, xW, beta), gS, fma(-gqW, qW, bq), gqN, x, q_prev);
        } else {
          const T xW = lx == 0 ? T(0) : x_prev;
          x = fma(-gW, xW, fma(-gS, xS, beta));
        }
      }
      P.xnew[gi] = x;
      x_prev = x;
      if (lane == BH - 1) {
        if (smem_prod) {
          ring[warp][lx % RING] = x;
          if (lx == 0) ring_tw[warp] = tw;
        } else if (gmem_prod && lx == 0) {
          P.twin_hand[slab_g] = tw;
        }
      }
    }
    // ---- publish progress of the top row (lane 31, column s-31)
    if (has_cons && lane == BH - 1) {
      const int lx31 = s - (BH - 1);
      if (lx31 >= 0 && lx31 < w && ((lx31 + 1) % CH == 0 || lx31 == w - 1)) {
        if (smem_prod) {
          __threadfence_block();
          ((volatile int*)prod)[warp] = lx31 + 1;
        } else {
          st_release(&P.flags[slab_g], (unsigned)(lx31 + 1));
        }
      }
    }
  }
}

// Algorithmic bytes of one sweep: each coefficient and vector value the
// sweep needs, read or written once per cell (halo and twin re-reads and
// old-value neighbour reads not counted).
template <class T, class TC, int KIND>
double sweep_bytes(int64_t N) {
  int coefs = 0, vecs = 0;
  if (KIND == KIND_SOR) { coefs = 5; vecs = 3; }          // inv, 4 c ; b, u_old, u_new
  else if (KIND == KIND_TRI_SCALED) { coefs = 3; vecs = 2; }  // inv, 2 c ; r, x
  else if (KIND == KIND_TRI_UNIT) { coefs = 2; vecs = 2; }    // 2 c ; r, x
  else { return 6.0 * 8.0 * (double)N; }                    // factor: 5 entries of A, d~
  return (double)N * (coefs * (double)sizeof(TC) + vecs * (double)sizeof(T));
}

template <class T, class TC, int KIND>
ndiag_status run(Handle* h, const SweepP<T, TC>& P, unsigned nslabs) {
  if (P.use_ticket) {
    ND_CUDA(cudaMemsetAsync(h->sync, 0, h->sync_bytes, h->stream));
  }
  const int slot = prof_begin(h);
  ++h->launches;
  ++h->sweep_launches;
  sweep2d_kernel<T, TC, KIND><<<nslabs, NW * 32, 0, h->stream>>>(P);
  ND_CUDA(cudaGetLastError());
  prof_end(h, slot, sweep_bytes<T, TC, KIND>((int64_t)P.nx * P.ny));
  return NDIAG_OK;
}

template <class T, class TC>
ndiag_status fill_and_run(Handle* h, int kind, int mode, int64_t t, const double* omega,
                          const ScaledSet& set, const void* rhs, const void* xold, void* xnew,
                          double beta_scale = 1.0, bool reverse_interior = false) {
  SweepP<T, TC> P{};
  P.bscale = (T)beta_scale;
  P.rev = reverse_interior ? 1 : 0;
  P.nx = (int)h->n[0];
  P.ny = (int)h->n[1];
  const bool nat = mode == NDIAG_NATURAL || mode == MODE_NATURAL_REV;
  const int px = nat ? 1 : h->sub[0], py = nat ? 1 : h->sub[1];
  P.sx = Split{px, P.nx / px, P.nx % px};
  P.sy = Split{py, P.ny / py, P.ny % py};
  P.base = nat ? (mode == MODE_NATURAL_REV ? 3 : 0) : base_corner(2, t);
  P.coupled = (nat || reverse_interior) ? 0 : 1;
  const int hmax = P.sy.len(0);
  const int bands = (hmax + BH - 1) / BH;
  P.spp = (bands + NW - 1) / NW;
  P.use_ticket = P.spp > 1;
  const size_t N = (size_t)h->N;
  const TC* base = (const TC*)set.base;
  P.inv = base;
  for (int e = 0; e < 4; ++e) P.c[e] = base + (size_t)(1 + e) * N;
  P.rhs = (const T*)rhs;
  P.xold = (const T*)xold;
  P.xnew = (T*)xnew;
  P.A = h->A64;
  for (int k = 0; k < 4; ++k) P.om[k] = omega ? (T)(nat ? omega[0] : omega[k]) : T(1);
  const unsigned nslabs = (unsigned)(px * py * P.spp);
  if (P.use_ticket) {
    const size_t need = sizeof(unsigned) * (1 + nslabs);
    const size_t need_tw = sizeof(T) * nslabs;
    if (need > h->sync_bytes) {
      if (h->sync) dev_free(h->sync, h->sync_bytes, h->stream);
      h->sync = (unsigned*)dev_alloc(need, h->stream);
      h->sync_bytes = h->sync ? need : 0;
      if (!h->sync) return NDIAG_ENOMEM;
    }
    if (need_tw > h->twin_hand_bytes) {
      if (h->twin_hand) dev_free(h->twin_hand, h->twin_hand_bytes, h->stream);
      h->twin_hand = dev_alloc(need_tw, h->stream);
      h->twin_hand_bytes = h->twin_hand ? need_tw : 0;
      if (!h->twin_hand) return NDIAG_ENOMEM;
    }
    P.ticket = h->sync;
    P.flags = h->sync + 1;
    P.twin_hand = (T*)h->twin_hand;
  }
  P.st = h->status;
  switch (kind) {
    case KIND_SOR: return run<T, TC, KIND_SOR>(h, P, nslabs);
    case KIND_TRI_SCALED: return run<T, TC, KIND_TRI_SCALED>(h, P, nslabs);
    case KIND_TRI_UNIT: return run<T, TC, KIND_TRI_UNIT>(h, P, nslabs);
    case KIND_FACTOR: return run<T, TC, KIND_FACTOR>(h, P, nslabs);
  }
  return NDIAG_EINVAL;
}

}  // namespace

ndiag_status launch_sweep2d_ex(Handle* h, int kind, int mode, int64_t t, const double* omega,
                               const ScaledSet& set, const void* rhs, const void* xold, void* xnew,
                               double beta_scale, bool rev) {
  const ndiag_status st = launch_sweep2d_staged(h, kind, mode, t, omega, set, rhs, xold, xnew, beta_scale, rev);
  if (st != NDIAG_EINVAL) return st;
  switch (h->precision) {
    case NDIAG_FP64:
      return fill_and_run<double, double>(h, kind, mode, t, omega, set, rhs, xold, xnew, beta_scale, rev);
    case NDIAG_FP32:
      return fill_and_run<float, float>(h, kind, mode, t, omega, set, rhs, xold, xnew, beta_scale, rev);
    case NDIAG_FP32_D16:
      return fill_and_run<float, __half>(h, kind, mode, t, omega, set, rhs, xold, xnew, beta_scale, rev);
  }
  return NDIAG_EINVAL;
}

ndiag_status launch_sweep2d(Handle* h, int kind, int mode, int64_t t, const double* omega,
                            const ScaledSet& set, const void* rhs, const void* xold, void* xnew) {
  return launch_sweep2d_ex(h, kind, mode, t, omega, set, rhs, xold, xnew, 1.0, false);
}

namespace {

// A triangular sweep (KIND_TRI_SCALED / KIND_TRI_UNIT, unit relaxation) whose
// slab hand-off words live in caller-provided device memory instead of the
// handle's lazily allocated buffers. Allocates nothing.
template <class T, class TC>
ndiag_status tri_sweep_in_scratch(Handle* h, int kind, int mode, int64_t t, const ScaledSet& set,
                                  const void* rhs, void* xnew, unsigned* sync, size_t sync_bytes,
                                  void* twin, size_t twin_bytes) {
  SweepP<T, TC> P{};
  P.bscale = T(1);
  P.rev = 0;
  P.nx = (int)h->n[0];
  P.ny = (int)h->n[1];
  const bool nat = mode == NDIAG_NATURAL || mode == MODE_NATURAL_REV;
  const int px = nat ? 1 : h->sub[0], py = nat ? 1 : h->sub[1];
  P.sx = Split{px, P.nx / px, P.nx % px};
  P.sy = Split{py, P.ny / py, P.ny % py};
  P.base = nat ? (mode == MODE_NATURAL_REV ? 3 : 0) : base_corner(2, t);
  P.coupled = nat ? 0 : 1;
  const int bands = (P.sy.len(0) + BH - 1) / BH;
  P.spp = (bands + NW - 1) / NW;
  P.use_ticket = P.spp > 1;
  const size_t N = (size_t)h->N;
  const TC* base = (const TC*)set.base;
  P.inv = base;
  for (int e = 0; e < 4; ++e) P.c[e] = base + (size_t)(1 + e) * N;
  P.rhs = (const T*)rhs;
  P.xold = nullptr;
  P.xnew = (T*)xnew;
  P.A = h->A64;
  for (int k = 0; k < 4; ++k) P.om[k] = T(1);
  const unsigned nslabs = (unsigned)(px * py * P.spp);
  if (P.use_ticket) {
    const size_t need = sizeof(unsigned) * (1 + (size_t)nslabs);
    if (need > sync_bytes || sizeof(T) * (size_t)nslabs > twin_bytes) {
      set_error("ilu0_apply_noalloc: the subdomain split needs more than 64 Ki hand-off words");
      return NDIAG_EINVAL;
    }
    ND_CUDA(cudaMemsetAsync(sync, 0, need, h->stream));  // hand-off words start at zero
    P.ticket = sync;
    P.flags = sync + 1;
    P.twin_hand = (T*)twin;
  }
  P.st = h->status;
  ++h->launches;
  ++h->sweep_launches;
  if (kind == KIND_TRI_SCALED)
    sweep2d_kernel<T, TC, KIND_TRI_SCALED><<<nslabs, NW * 32, 0, h->stream>>>(P);
  else
    sweep2d_kernel<T, TC, KIND_TRI_UNIT><<<nslabs, NW * 32, 0, h->stream>>>(P);
  ND_CUDA(cudaGetLastError());
  return NDIAG_OK;
}

}  // namespace

ndiag_status launch_tri_sweep2d_scratch(Handle* h, int kind, int mode, int64_t t, const ScaledSet& set,
                                        const void* rhs, void* xnew, unsigned* sync, size_t sync_bytes,
                                        void* twin, size_t twin_bytes) {
  if (kind != KIND_TRI_SCALED && kind != KIND_TRI_UNIT) return NDIAG_EINVAL;
  switch (h->precision) {
    case NDIAG_FP64:
      return tri_sweep_in_scratch<double, double>(h, kind, mode, t, set, rhs, xnew, sync, sync_bytes, twin,
                                                  twin_bytes);
    case NDIAG_FP32:
      return tri_sweep_in_scratch<float, float>(h, kind, mode, t, set, rhs, xnew, sync, sync_bytes, twin,
                                                twin_bytes);
    case NDIAG_FP32_D16:
      return tri_sweep_in_scratch<float, __half>(h, kind, mode, t, set, rhs, xnew, sync, sync_bytes, twin,
                                                 twin_bytes);
  }
  return NDIAG_EINVAL;
}

// d~ of the decomposed (or natural) ILU(0), written to `out` (fp64, N): the
// same wavefront without interface coupling, since a mutual pair contributes
// no elimination term (Sec. 5).
ndiag_status launch_ilu_factor2d_into(Handle* h, int mode, double* out) {
  ScaledSet dummy;
  dummy.base = h->A64;  // unused by the factor kind
  return fill_and_run<double, double>(h, KIND_FACTOR, mode, fwd_phase(2), nullptr, dummy, nullptr,
                                      nullptr, out);
}

}  // namespace nd
