// Vector kernels of the Krylov drivers: stencil SpMV, residual, fused
// updates, and dot products with a deterministic two-level reduction (fixed
// grid, fixed order; the last block to finish sums the block partials in
// index order, so a result does not depend on scheduling).
#include <initializer_list>

#include "blas.h"

namespace nd {

namespace {
constexpr int BT = 256;  // threads per block
constexpr int BPS = 4;   // resident blocks per SM the kernels are bounded for (64 registers)
// Elements per thread per loop trip. Each trip issues all its loads before any
// arithmetic or store, so a thread keeps U loads per stream in flight; with
// BPS x BT threads per SM that is enough to cover HBM latency on GB300.
constexpr int U = 4;
constexpr int BPS_STENCIL = 3;  // the stencil kernels hold ten loads per cell, two cells per thread

#define ND_STREAM_LOOP(N)                                                              \
  for (int64_t base = (int64_t)blockIdx.x * (BT * U) + threadIdx.x; base < (N);        \
       base += (int64_t)gridDim.x * (BT * U))

__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < BT / 32; ++k) r += sh[k];
  __syncthreads();
  return r;  // valid in thread 0
}

// Writes NV block partials; the last block sums them into res[0..NV).
template <int NV>
__device__ void finish_reduce(const double (&v)[NV], Reduce R) {
  __shared__ double sh[BT / 32];
  __shared__ bool last;
  double tot[NV];
  for (int k = 0; k < NV; ++k) tot[k] = block_sum(v[k], sh);
  if (threadIdx.x == 0) {
    for (int k = 0; k < NV; ++k) R.part[(size_t)k * gridDim.x + blockIdx.x] = tot[k];
    __threadfence();
    last = atomicAdd(R.counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last) {
    __threadfence();
    for (int k = 0; k < NV; ++k) {
      double acc = 0.0;
      for (unsigned b = threadIdx.x; b < gridDim.x; b += BT) acc += __ldcg(R.part + (size_t)k * gridDim.x + b);
      acc = block_sum(acc, sh);
      if (threadIdx.x == 0) R.res[k] = acc;
    }
    if (threadIdx.x == 0) *R.counter = 0;
  }
}

struct Geo {
  int nx, ny, nz, stencil;
  int64_t N;
};

// (A x)_i for a structured stencil; the matrix A is diagonal-major (s, N).
// IDX is the index type of the cell coordinates: 32-bit division whenever the
// grid has fewer than 2^31 cells.
template <class T, class TA, class IDX>
__device__ __forceinline__ T stencil_apply(const Geo& g, const TA* __restrict__ A, const T* __restrict__ x,
                                           int64_t i) {
  const IDX ii = (IDX)i, nx = (IDX)g.nx, ny = (IDX)g.ny;
  const IDX rest = ii / nx;
  const int cx = (int)(ii - rest * nx);
  const IDX rz = rest / ny;
  const int cy = (int)(rest - rz * ny);
  const int cz = (int)rz;
  const int64_t N = g.N;
  T acc = (T)A[i] * x[i];
  if (cx > 0) acc = fma((T)A[N + i], x[i - 1], acc);
  if (cx + 1 < g.nx) acc = fma((T)A[2 * N + i], x[i + 1], acc);
  if (cy > 0) acc = fma((T)A[3 * N + i], x[i - g.nx], acc);
  if (cy + 1 < g.ny) acc = fma((T)A[4 * N + i], x[i + g.nx], acc);
  if (g.stencil == 7) {
    const int64_t pl = (int64_t)g.nx * g.ny;
    if (cz > 0) acc = fma((T)A[5 * N + i], x[i - pl], acc);
    if (cz + 1 < g.nz) acc = fma((T)A[6 * N + i], x[i + pl], acc);
  } else if (g.stencil == 9) {
    if (cx > 0 && cy > 0) acc = fma((T)A[5 * N + i], x[i - g.nx - 1], acc);
    if (cx + 1 < g.nx && cy > 0) acc = fma((T)A[6 * N + i], x[i - g.nx + 1], acc);
    if (cx > 0 && cy + 1 < g.ny) acc = fma((T)A[7 * N + i], x[i + g.nx - 1], acc);
    if (cx + 1 < g.nx && cy + 1 < g.ny) acc = fma((T)A[8 * N + i], x[i + g.nx + 1], acc);
  }
  return acc;
}

// y = A x ; ND = 1: partial (w, y); ND = 2: also (y, y). Two cells per thread
// per trip (the stencil reads ten values per cell).
template <class T, class TA, int ND, class IDX>
__global__ void __launch_bounds__(BT, BPS_STENCIL) spmv_kernel(Geo g, const TA* __restrict__ A, const T* __restrict__ x,
                                                       T* __restrict__ y, const T* __restrict__ w, Reduce R) {
  constexpr int V = 2;
  double d0 = 0.0, d1 = 0.0;
  for (int64_t base = (int64_t)blockIdx.x * (BT * V) + threadIdx.x; base < g.N;
       base += (int64_t)gridDim.x * (BT * V)) {
    T v[V], wv[V];
#pragma unroll
    for (int u = 0; u < V; ++u) {
      const int64_t i = base + u * BT;
      if (i < g.N) {
        v[u] = stencil_apply<T, TA, IDX>(g, A, x, i);
        if (ND >= 1) wv[u] = w[i];
      }
    }
#pragma unroll
    for (int u = 0; u < V; ++u) {
      const int64_t i = base + u * BT;
      if (i < g.N) {
        y[i] = v[u];
        if (ND >= 1) d0 += (double)wv[u] * (double)v[u];
        if (ND >= 2) d1 += (double)v[u] * (double)v[u];
      }
    }
  }
  if (ND == 1) {
    double vv[1] = {d0};
    finish_reduce<1>(vv, R);
  } else if (ND == 2) {
    double vv[2] = {d0, d1};
    finish_reduce<2>(vv, R);
  }
}

template <class T>
struct Pair;
template <>
struct Pair<double> {
  using type = double2;
};
template <>
struct Pair<float> {
  using type = float2;
};

// 2D 5-point y = A x on cell pairs (i, i + 1), i even, nx even: the five
// diagonals, x, w and y move as pairs; x[i - 1] and x[i + 2] are single loads
// (L1 hits). ND as in spmv_kernel. Every thread keeps one pair's eleven
// loads in flight.
template <class T, int ND>
__global__ void __launch_bounds__(BT, BPS) spmv5_pair_kernel(int nx, int ny, int64_t N, const T* __restrict__ A,
                                                             const T* __restrict__ x, T* __restrict__ y,
                                                             const T* __restrict__ w, Reduce R) {
  using P2 = typename Pair<T>::type;
  const int64_t np = N / 2;
  const unsigned hx = (unsigned)nx / 2;
  const P2* A2 = reinterpret_cast<const P2*>(A);
  const P2* x2 = reinterpret_cast<const P2*>(x);
  const P2* w2 = reinterpret_cast<const P2*>(w);
  P2* y2 = reinterpret_cast<P2*>(y);
  const int64_t NP = np;  // pairs per diagonal
  double d0 = 0.0, d1 = 0.0;
  for (int64_t p = (int64_t)blockIdx.x * BT + threadIdx.x; p < np; p += (int64_t)gridDim.x * BT) {
    const unsigned row = (unsigned)p / hx;
    const int cx = 2 * (int)((unsigned)p - row * hx), cy = (int)row;
    const int64_t i = 2 * p;
    const P2 a0 = A2[p], aW = A2[NP + p], aE = A2[2 * NP + p], aS = A2[3 * NP + p], aN = A2[4 * NP + p];
    const P2 xc = x2[p];
    const bool hw = cx > 0, he = cx + 2 < nx, hs = cy > 0, hn = cy + 1 < ny;
    const T xw = hw ? x[i - 1] : T(0);
    const T xe = he ? x[i + 2] : T(0);
    P2 xs, xn, wv;
    if (hs) xs = x2[p - hx];
    if (hn) xn = x2[p + hx];
    if (ND >= 1) wv = w2[p];
    T v0 = a0.x * xc.x, v1 = a0.y * xc.y;
    if (hw) v0 = fma(aW.x, xw, v0);
    v1 = fma(aW.y, xc.x, v1);
    v0 = fma(aE.x, xc.y, v0);
    if (he) v1 = fma(aE.y, xe, v1);
    if (hs) {
      v0 = fma(aS.x, xs.x, v0);
      v1 = fma(aS.y, xs.y, v1);
    }
    if (hn) {
      v0 = fma(aN.x, xn.x, v0);
      v1 = fma(aN.y, xn.y, v1);
    }
    P2 out;
    out.x = v0;
    out.y = v1;
    y2[p] = out;
    if (ND >= 1) d0 += (double)wv.x * (double)v0 + (double)wv.y * (double)v1;
    if (ND >= 2) d1 += (double)v0 * (double)v0 + (double)v1 * (double)v1;
  }
  if (ND == 1) {
    double vv[1] = {d0};
    finish_reduce<1>(vv, R);
  } else if (ND == 2) {
    double vv[2] = {d0, d1};
    finish_reduce<2>(vv, R);
  }
}

// r = b - A x (fp64), ||r||^2
template <class TB, class IDX>
__global__ void __launch_bounds__(BT, BPS_STENCIL) residual_kernel(Geo g, const double* __restrict__ A,
                                                           const double* __restrict__ b,
                                                           const double* __restrict__ x, TB* __restrict__ r,
                                                           Reduce R) {
  constexpr int V = 2;
  double d = 0.0;
  for (int64_t base = (int64_t)blockIdx.x * (BT * V) + threadIdx.x; base < g.N;
       base += (int64_t)gridDim.x * (BT * V)) {
    double v[V];
#pragma unroll
    for (int u = 0; u < V; ++u) {
      const int64_t i = base + u * BT;
      if (i < g.N) v[u] = b[i] - stencil_apply<double, double, IDX>(g, A, x, i);
    }
#pragma unroll
    for (int u = 0; u < V; ++u) {
      const int64_t i = base + u * BT;
      if (i < g.N) {
        r[i] = (TB)v[u];
        d += v[u] * v[u];
      }
    }
  }
  double vv[1] = {d};
  finish_reduce<1>(vv, R);
}

// generic fused dots: up to 3 inner products (a_k, b_k)
template <class T, int NV>
__global__ void __launch_bounds__(BT, BPS) dots_kernel(int64_t N, const T* __restrict__ a0,
                                                       const T* __restrict__ b0, const T* __restrict__ a1,
                                                       const T* __restrict__ b1, const T* __restrict__ a2,
                                                       const T* __restrict__ b2, Reduce R) {
  double d[NV];
  for (int k = 0; k < NV; ++k) d[k] = 0.0;
  constexpr int U = NV > 2 ? 3 : (NV > 1 ? 4 : 8);
  ND_STREAM_LOOP(N) {
    T va[NV][U], vb[NV][U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = base + u * BT;
      if (i < N) {
        va[0][u] = a0[i], vb[0][u] = b0[i];
        if (NV > 1) va[1 % NV][u] = a1[i], vb[1 % NV][u] = b1[i];
        if (NV > 2) va[2 % NV][u] = a2[i], vb[2 % NV][u] = b2[i];
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (base + u * BT < N)
        for (int k = 0; k < NV; ++k) d[k] += (double)va[k][u] * (double)vb[k][u];
  }
  finish_reduce<NV>(d, R);
}

// ---- BiCGSTAB steps (scalars live in device memory) ----
// p = r + beta (p - om v),  beta = (rho/rho_old)(alpha/om)
// sp (optional) = inv .* p: the right-hand side of a forward sweep whose
// diagonal scaling is taken here (the pre-scaled ILU(0) apply)
template <class T>
__global__ void __launch_bounds__(BT, BPS) bicg_p_kernel(int64_t N, const T* __restrict__ r, T* __restrict__ p,
                                                         const T* __restrict__ v, const double* sc, int first,
                                                         const T* __restrict__ inv, T* __restrict__ sp) {
  if (sc[SC_DONE] != 0.0) return;  // the iteration has stopped
  const double rho = sc[SC_RHO], rho_old = sc[SC_RHO_OLD], alpha = sc[SC_ALPHA], om = sc[SC_OM];
  const double beta = first ? 0.0 : (rho / rho_old) * (alpha / om);
  constexpr int U = 4;  // three or four streams in
  ND_STREAM_LOOP(N) {
    T vr[U], vp[U], vv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = base + u * BT;
      if (i < N) {
        vr[u] = r[i];
        if (!first) vp[u] = p[i], vv[u] = v[i];
      }
    }
    T vi[U];
    if (sp) {
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (base + u * BT < N) vi[u] = inv[base + u * BT];
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = base + u * BT;
      if (i < N) {
        const T pv = first ? vr[u] : (T)((double)vr[u] + beta * ((double)vp[u] - om * (double)vv[u]));
        p[i] = pv;
        if (sp) sp[i] = vi[u] * pv;
      }
    }
  }
}
// s = r - alpha v, alpha = rho / (rh, v); ||s||^2
template <class T>
__global__ void __launch_bounds__(BT, BPS) bicg_s_kernel(int64_t N, const T* __restrict__ r,
                                                         const T* __restrict__ v, T* __restrict__ s,
                                                         const double* sc, Reduce R, const T* __restrict__ inv,
                                                         T* __restrict__ ss) {
  if (sc[SC_DONE] != 0.0) return;  // every block returns: the reduction is not touched
  const double alpha = sc[SC_RHO] / sc[SC_RV];
  double d = 0.0;
  constexpr int U = 4;  // two or three streams in
  ND_STREAM_LOOP(N) {
    T vr[U], vv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = base + u * BT;
      if (i < N) vr[u] = r[i], vv[u] = v[i];
    }
    T vi[U];
    if (ss) {
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (base + u * BT < N) vi[u] = inv[base + u * BT];
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = base + u * BT;
      if (i < N) {
        const T sv = (T)((double)vr[u] - alpha * (double)vv[u]);
        s[i] = sv;
        if (ss) ss[i] = vi[u] * sv;
        d += (double)sv * (double)sv;
      }
    }
  }
  double vv[1] = {d};
  finish_reduce<1>(vv, R);
}
// x += alpha ph + om sh ; r = s - om t ; ||r||^2, (rh, r)
template <class T>
__global__ void __launch_bounds__(BT, BPS) bicg_xr_kernel(int64_t N, T* __restrict__ x, const T* __restrict__ ph,
                                                          const T* __restrict__ sh, T* __restrict__ r,
                                                          const T* __restrict__ s, const T* __restrict__ t,
                                                          const T* __restrict__ rh, const double* sc, Reduce R) {
  // Breakdown of the first half step (rho = 0, (rh, v) = 0 or a non-finite s)
  // leaves x and r as they are; the host reports it. A first half step that
  // already meets the tolerance (||s||^2 <= tol^2) takes om = 0: x += alpha ph
  // and r = s, the solution of the half step.
  if (sc[SC_DONE] != 0.0) return;
  const double rho = sc[SC_RHO], rv = sc[SC_RV], ss = sc[SC_SS];
  if (rho == 0.0 || rv == 0.0 || !isfinite(ss)) return;
  const double alpha = rho / rv;
  const double tt = sc[SC_TT];
  const double om = (ss <= sc[SC_TOL2] || tt == 0.0) ? 0.0 : sc[SC_TS] / tt;
  double d0 = 0.0, d1 = 0.0;
  constexpr int U = 2;  // six streams
  ND_STREAM_LOOP(N) {
    T vx[U], vph[U], vsh[U], vs[U], vt[U], vrh[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = base + u * BT;
      if (i < N) vx[u] = x[i], vph[u] = ph[i], vsh[u] = sh[i], vs[u] = s[i], vt[u] = t[i], vrh[u] = rh[i];
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = base + u * BT;
      if (i < N) {
        x[i] = (T)((double)vx[u] + alpha * (double)vph[u] + om * (double)vsh[u]);
        const T rv = (T)((double)vs[u] - om * (double)vt[u]);
        r[i] = rv;
        d0 += (double)rv * (double)rv;
        d1 += (double)vrh[u] * (double)rv;
      }
    }
  }
  double vv[2] = {d0, d1};
  finish_reduce<2>(vv, R);
}
// x += alpha ph  (exit at the half step)
template <class T>
__global__ void __launch_bounds__(BT, BPS) axpy_alpha_kernel(int64_t N, T* __restrict__ x,
                                                             const T* __restrict__ ph, const double* sc) {
  const double alpha = sc[SC_RHO] / sc[SC_RV];
  ND_STREAM_LOOP(N) {
    T vx[U], vp[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = base + u * BT;
      if (i < N) vx[u] = x[i], vp[u] = ph[i];
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = base + u * BT;
      if (i < N) x[i] = (T)((double)vx[u] + alpha * (double)vp[u]);
    }
  }
}

// ---- PCG steps ----
// x += alpha p ; r -= alpha q ; ||r||^2 ; alpha = rz / (p, q)
template <class T>
__global__ void __launch_bounds__(BT, BPS) cg_xr_kernel(int64_t N, T* __restrict__ x, const T* __restrict__ p,
                                                        T* __restrict__ r, const T* __restrict__ q,
                                                        const double* sc, Reduce R) {
  if (sc[SC_DONE] != 0.0) return;
  const double alpha = sc[SC_RZ] / sc[SC_PQ];
  double d = 0.0;
  constexpr int U = 4;  // four streams
  ND_STREAM_LOOP(N) {
    T vx[U], vp[U], vr[U], vq[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = base + u * BT;
      if (i < N) vx[u] = x[i], vp[u] = p[i], vr[u] = r[i], vq[u] = q[i];
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = base + u * BT;
      if (i < N) {
        x[i] = (T)((double)vx[u] + alpha * (double)vp[u]);
        const T rv = (T)((double)vr[u] - alpha * (double)vq[u]);
        r[i] = rv;
        d += (double)rv * (double)rv;
      }
    }
  }
  double vv[1] = {d};
  finish_reduce<1>(vv, R);
}
// p = z + beta p, beta = rz_new / rz ; first: p = z
template <class T>
__global__ void __launch_bounds__(BT, BPS) cg_p_kernel(int64_t N, const T* __restrict__ z, T* __restrict__ p,
                                                       const double* sc, int first) {
  if (sc[SC_DONE] != 0.0) return;
  const double beta = first ? 0.0 : sc[SC_RZ_NEW] / sc[SC_RZ];
  constexpr int U = 8;  // two streams in
  ND_STREAM_LOOP(N) {
    T vz[U], vp[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = base + u * BT;
      if (i < N) {
        vz[u] = z[i];
        if (!first) vp[u] = p[i];
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = base + u * BT;
      if (i < N) p[i] = first ? vz[u] : (T)((double)vz[u] + beta * (double)vp[u]);
    }
  }
}

__global__ void copy_scalar_kernel(double* sc, int dst, int src) {
  if (sc[SC_DONE] == 0.0) sc[dst] = sc[src];
}

template <class TD, class TS>
__global__ void __launch_bounds__(BT, BPS) convert_kernel(int64_t N, const TS* __restrict__ s, TD* __restrict__ d) {
  ND_STREAM_LOOP(N) {
    TS v[U];
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (base + u * BT < N) v[u] = s[base + u * BT];
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (base + u * BT < N) d[base + u * BT] = (TD)v[u];
  }
}
__global__ void __launch_bounds__(BT, BPS) add_to_kernel(int64_t N, double* __restrict__ x,
                                                         const float* __restrict__ e) {
  ND_STREAM_LOOP(N) {
    double vx[U];
    float ve[U];
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (base + u * BT < N) vx[u] = x[base + u * BT], ve[u] = e[base + u * BT];
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (base + u * BT < N) x[base + u * BT] = vx[u] + (double)ve[u];
  }
}
template <class T>
__global__ void __launch_bounds__(BT, BPS) scale_kernel(int64_t N, T* __restrict__ x, double f) {
  ND_STREAM_LOOP(N) {
    T v[U];
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (base + u * BT < N) v[u] = x[base + u * BT];
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (base + u * BT < N) x[base + u * BT] = (T)((double)v[u] * f);
  }
}
template <class T>
__global__ void __launch_bounds__(BT, BPS) mul_kernel(int64_t N, const double* __restrict__ A0,
                                                      const T* __restrict__ x, T* __restrict__ y) {
  ND_STREAM_LOOP(N) {
    double va[U];
    T vx[U];
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (base + u * BT < N) va[u] = A0[base + u * BT], vx[u] = x[base + u * BT];
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (base + u * BT < N) y[base + u * BT] = (T)(va[u] * (double)vx[u]);
  }
}

Geo geo(const Handle* h) {
  return Geo{(int)h->n[0], (int)h->n[1], (int)h->n[2], h->stencil, h->N};
}
}  // namespace

// One grid size for every vector kernel of a handle (a fixed function of N and
// the SM count, so the reductions sum in a fixed order): BPS resident blocks
// per SM, fewer when the vector is short.
int grid_blocks(const Handle* h) {
  const int64_t need = (h->N + BT * 2 - 1) / (BT * 2);
  const int64_t cap = (int64_t)h->sm_count * BPS;
  return (int)(need < cap ? (need < 1 ? 1 : need) : cap);
}

Reduce reduce_slot(Handle* h, int slot) {
  Reduce R;
  const int G = grid_blocks(h);
  R.part = h->red + RED_RES + (size_t)slot * 4 * G;  // 4 values per slot region
  R.counter = (unsigned*)(h->red) + 2 * slot;
  R.res = h->red + SC_BASE;  // overridden by callers
  return R;
}

size_t reduce_bytes(const Handle* h) {
  return sizeof(double) * (RED_RES + (size_t)RED_SLOTS * 4 * grid_blocks(h));
}

#define LAUNCH_G(grid, kern, ...)                       \
  do {                                                  \
    ++h->launches;                                      \
    kern<<<(grid), BT, 0, h->stream>>>(__VA_ARGS__);    \
    ND_CUDA(cudaGetLastError());                        \
  } while (0)
#define LAUNCH(kern, ...) LAUNCH_G(grid_blocks(h), kern, __VA_ARGS__)

// cell coordinates in 32-bit arithmetic when the grid allows it
bool small_index(const Handle* h) { return h->N < ((int64_t)1 << 31); }

#define ND_UNPAREN(...) __VA_ARGS__
// the stencil kernels: at most BPS_STENCIL blocks per SM (a subset of the
// partial slots of grid_blocks)
int stencil_blocks(const Handle* h) {
  const int g = grid_blocks(h), cap = h->sm_count * BPS_STENCIL;
  return g < cap ? g : cap;
}
#define LAUNCH_IDX(kern, targs, ...)                                                                      \
  do {                                                                                                    \
    if (small_index(h)) LAUNCH_G(stencil_blocks(h), (kern<ND_UNPAREN targs, uint32_t>), __VA_ARGS__);     \
    else LAUNCH_G(stencil_blocks(h), (kern<ND_UNPAREN targs, uint64_t>), __VA_ARGS__);                    \
  } while (0)

ndiag_status spmv64(Handle* h, const double* x, double* y) {
  Reduce R{};
  LAUNCH_IDX(spmv_kernel, (double, double, 0), geo(h), h->A64, x, y, (const double*)nullptr, R);
  return NDIAG_OK;
}

// 2D 5-point grids with even nx and pair-aligned vectors take the pair kernel
template <class T>
bool pair_ok(const Handle* h, const void* A, std::initializer_list<const void*> v) {
  if (h->stencil != 5 || h->n[2] != 1 || (h->n[0] & 1) || !small_index(h)) return false;
  if ((uintptr_t)A % (2 * sizeof(T))) return false;
  for (const void* p : v)
    if (p && (uintptr_t)p % (2 * sizeof(T))) return false;
  return true;
}

template <class T>
ndiag_status spmv_dot(Handle* h, const T* x, T* y, const T* w, double* res, int slot, bool two) {
  Reduce R = reduce_slot(h, slot);
  R.res = res;
  const T* A = sizeof(T) == 8 ? (const T*)h->A64 : (const T*)h->Alo;
  if (pair_ok<T>(h, A, {x, y, w})) {
    if (two) LAUNCH((spmv5_pair_kernel<T, 2>), (int)h->n[0], (int)h->n[1], h->N, A, x, y, w, R);
    else LAUNCH((spmv5_pair_kernel<T, 1>), (int)h->n[0], (int)h->n[1], h->N, A, x, y, w, R);
    return NDIAG_OK;
  }
  if (sizeof(T) == 8) {
    if (two) LAUNCH_IDX(spmv_kernel, (T, double, 2), geo(h), h->A64, x, y, w, R);
    else LAUNCH_IDX(spmv_kernel, (T, double, 1), geo(h), h->A64, x, y, w, R);
  } else {
    if (two) LAUNCH_IDX(spmv_kernel, (T, float, 2), geo(h), (const float*)h->Alo, x, y, w, R);
    else LAUNCH_IDX(spmv_kernel, (T, float, 1), geo(h), (const float*)h->Alo, x, y, w, R);
  }
  return NDIAG_OK;
}
template <class T>
ndiag_status spmv_any(Handle* h, const T* x, T* y) {
  Reduce R{};
  if (sizeof(T) == 8)
    LAUNCH_IDX(spmv_kernel, (T, double, 0), geo(h), h->A64, x, y, (const T*)nullptr, R);
  else
    LAUNCH_IDX(spmv_kernel, (T, float, 0), geo(h), (const float*)h->Alo, x, y, (const T*)nullptr, R);
  return NDIAG_OK;
}

ndiag_status residual64(Handle* h, const double* b, const double* x, double* r, double* res) {
  Reduce R = reduce_slot(h, 0);
  R.res = res;
  LAUNCH_IDX(residual_kernel, (double), geo(h), h->A64, b, x, r, R);
  return NDIAG_OK;
}
ndiag_status residual64_to32(Handle* h, const double* b, const double* x, float* r, double* res) {
  Reduce R = reduce_slot(h, 0);
  R.res = res;
  LAUNCH_IDX(residual_kernel, (float), geo(h), h->A64, b, x, r, R);
  return NDIAG_OK;
}

template <class T>
ndiag_status dots(Handle* h, int nv, const T* a0, const T* b0, const T* a1, const T* b1, const T* a2,
                  const T* b2, double* res, int slot) {
  Reduce R = reduce_slot(h, slot);
  R.res = res;
  if (nv == 1) LAUNCH((dots_kernel<T, 1>), h->N, a0, b0, a1, b1, a2, b2, R);
  else if (nv == 2) LAUNCH((dots_kernel<T, 2>), h->N, a0, b0, a1, b1, a2, b2, R);
  else LAUNCH((dots_kernel<T, 3>), h->N, a0, b0, a1, b1, a2, b2, R);
  return NDIAG_OK;
}

template <class T>
ndiag_status bicg_p(Handle* h, const T* r, T* p, const T* v, const double* sc, int first, const T* inv, T* sp) {
  LAUNCH((bicg_p_kernel<T>), h->N, r, p, v, sc, first, inv, sp);
  return NDIAG_OK;
}
template <class T>
ndiag_status bicg_s(Handle* h, const T* r, const T* v, T* s, double* sc, const T* inv, T* ss) {
  Reduce R = reduce_slot(h, 1);
  R.res = sc + SC_SS;
  LAUNCH((bicg_s_kernel<T>), h->N, r, v, s, sc, R, inv, ss);
  return NDIAG_OK;
}
template <class T>
ndiag_status bicg_xr(Handle* h, T* x, const T* ph, const T* sh, T* r, const T* s, const T* t, const T* rh,
                     double* sc) {
  Reduce R = reduce_slot(h, 2);
  R.res = sc + SC_RR;  // writes SC_RR, SC_RR+1 (= SC_RHO_NEXT)
  LAUNCH((bicg_xr_kernel<T>), h->N, x, ph, sh, r, s, t, rh, sc, R);
  return NDIAG_OK;
}
template <class T>
ndiag_status axpy_alpha(Handle* h, T* x, const T* ph, const double* sc) {
  LAUNCH((axpy_alpha_kernel<T>), h->N, x, ph, sc);
  return NDIAG_OK;
}
template <class T>
ndiag_status cg_xr(Handle* h, T* x, const T* p, T* r, const T* q, double* sc) {
  Reduce R = reduce_slot(h, 1);
  R.res = sc + SC_RR;
  LAUNCH((cg_xr_kernel<T>), h->N, x, p, r, q, sc, R);
  return NDIAG_OK;
}
template <class T>
ndiag_status cg_p(Handle* h, const T* z, T* p, const double* sc, int first) {
  LAUNCH((cg_p_kernel<T>), h->N, z, p, sc, first);
  return NDIAG_OK;
}
ndiag_status copy_scalar(Handle* h, double* sc, int dst, int src) {
  ++h->launches;
  copy_scalar_kernel<<<1, 1, 0, h->stream>>>(sc, dst, src);
  ND_CUDA(cudaGetLastError());
  return NDIAG_OK;
}
ndiag_status to32(Handle* h, const double* s, float* d) {
  LAUNCH((convert_kernel<float, double>), h->N, s, d);
  return NDIAG_OK;
}
ndiag_status add_to(Handle* h, double* x, const float* e) {
  LAUNCH(add_to_kernel, h->N, x, e);
  return NDIAG_OK;
}
template <class T>
ndiag_status scale(Handle* h, T* x, double f) {
  LAUNCH((scale_kernel<T>), h->N, x, f);
  return NDIAG_OK;
}
template <class T>
ndiag_status mul_diag(Handle* h, const T* x, T* y) {
  LAUNCH((mul_kernel<T>), h->N, h->A64, x, y);
  return NDIAG_OK;
}

#define INST(T)                                                                                         \
  template ndiag_status spmv_dot<T>(Handle*, const T*, T*, const T*, double*, int, bool);                    \
  template ndiag_status spmv_any<T>(Handle*, const T*, T*);                                            \
  template ndiag_status dots<T>(Handle*, int, const T*, const T*, const T*, const T*, const T*,         \
                                const T*, double*, int);                                               \
  template ndiag_status bicg_p<T>(Handle*, const T*, T*, const T*, const double*, int, const T*, T*);  \
  template ndiag_status bicg_s<T>(Handle*, const T*, const T*, T*, double*, const T*, T*);             \
  template ndiag_status bicg_xr<T>(Handle*, T*, const T*, const T*, T*, const T*, const T*, const T*,  \
                                   double*);                                                           \
  template ndiag_status axpy_alpha<T>(Handle*, T*, const T*, const double*);                           \
  template ndiag_status cg_xr<T>(Handle*, T*, const T*, T*, const T*, double*);                        \
  template ndiag_status cg_p<T>(Handle*, const T*, T*, const double*, int);                            \
  template ndiag_status scale<T>(Handle*, T*, double);                                                 \
  template ndiag_status mul_diag<T>(Handle*, const T*, T*);
INST(double)
INST(float)

}  // namespace nd
