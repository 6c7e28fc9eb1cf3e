// Symmetric SSOR apply on 2D 5-point matrices (Sec. 2: SSOR = a sweep and its
// reverse; Sec. 5), SPD form for CG:
//     z = w(2-w) (D + w L_J^T)^-1 D (D + w L_J)^-1 r .
//
// Forward half: the ordinary decomposed sweep of the forward phase with the
// factor w(2-w) folded into beta.
// Backward half, a transposed solve: cell i depends on every j with i in J_j.
// Inside a subdomain that is the reversed wavefront (run by the sweep kernel
// in the reversed frame, without twins, leaving out the start lines that border
// coupled interfaces). The coupled pairs along an interface depend on the
// interior cells of both subdomains and are solved afterwards, from the far
// end of the interface back to its start vertex, one warp per interface;
// the four start corners at a vertex form the 4x4 system of Eq. (2d:sor4b4),
// solved by whichever of the vertex's four interface chains finishes last
// (arrival counter, no waiting).
#include <algorithm>
#include <cstring>
#include <vector>

#include "internal.h"

namespace nd {
namespace {

template <class T, class TC>
__device__ __forceinline__ T ldc(const TC* p) {
  return (T)__ldcg(p);
}
template <>
__device__ __forceinline__ float ldc<float, __half>(const __half* p) {
  return __half2float(__ldcg(p));
}

template <class T, class TC>
struct EdgeP {
  int nx, ny;
  Split sx, sy;
  int base;
  const TC* cT[4];  // transposed scaled entries, W E S N
  const T* w;       // right-hand side of the backward solve
  T* z;
  T om;
  unsigned* vcount;
};

template <class T, class TC>
__device__ __forceinline__ T coef(const EdgeP<T, TC>& P, int e, int64_t i) {
  return P.om * ldc<T, TC>(P.cT[e] + i);
}

template <class T>
__device__ __forceinline__ void corner_solve(const T h[4], const T gx[4], const T gy[4], T x[4]) {
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

// 4x4 corner at interior vertex (vx, vy): slots k = (X + (k&1), Y + (k>>1)).
template <class T, class TC>
__device__ void solve_vertex(const EdgeP<T, TC>& P, int vx, int vy) {
  const int X = P.sx.lo(vx + 1) - 1, Y = P.sy.lo(vy + 1) - 1;
  T hh[4], gx[4], gy[4], xx[4];
  int64_t idx[4];
  for (int k = 0; k < 4; ++k) {
    const int bx = k & 1, by = k >> 1;
    const int cx = X + bx, cy = Y + by;
    const int64_t i = (int64_t)cy * P.nx + cx;
    idx[k] = i;
    T hv = __ldcg(P.w + i);
    // downstream neighbours inside the cell's own subdomain (away from the vertex)
    const int ix = vx + bx, iy = vy + by;
    if (P.sx.len(ix) >= 2) {
      const int e = bx ? 1 : 0;  // E for the right column, W for the left one
      hv = fma(-coef(P, e, i), __ldcg(P.z + i + (bx ? 1 : -1)), hv);
    }
    if (P.sy.len(iy) >= 2) {
      const int e = by ? 3 : 2;
      hv = fma(-coef(P, e, i), __ldcg(P.z + i + (by ? P.nx : -P.nx)), hv);
    }
    hh[k] = hv;
    gx[k] = coef(P, bx ? 0 : 1, i);  // towards slot k^1
    gy[k] = coef(P, by ? 2 : 3, i);  // towards slot k^2
  }
  corner_solve(hh, gx, gy, xx);
  for (int k = 0; k < 4; ++k) P.z[idx[k]] = xx[k];
}

// Chains are run by one warp each: lanes load the inputs of 32 consecutive
// pairs at once (right-hand side, the interior neighbour terms, the couplings
// and 1/det of every 2x2 pair system), then lane 0 runs the recurrence over
// them, three dependent operations a pair, and the warp stores the results.
constexpr int ELN = 32;            // lanes per chain
constexpr int ETH = 128;           // threads per block: 4 chains
constexpr int ECH = ETH / ELN;

// per-warp staging of one chunk of a chain
template <class T>
struct Chunk {
  T hp[ELN], hq[ELN], a[ELN], b[ELN], gab[ELN], gba[ELN], idet[ELN];
};

// Pair k of a chain (k = 0 at the far end): cells ip, iq of the pair, the
// entries towards the previous pair (k - 1), between the two cells, and the
// interior neighbour terms, staged into slot j of the chunk.
template <class T, class TC>
__device__ __forceinline__ void stage_pair(const EdgeP<T, TC>& P, const TC* const (&c)[5], Chunk<T>& C, int j,
                                           int k, int64_t ip, int64_t iq, int64_t dip, int64_t diq, bool in_p,
                                           bool in_q) {
  T hp = __ldcg(P.w + ip), hq = __ldcg(P.w + iq);
  if (in_p) hp = fma(-(P.om * ldc<T, TC>(c[3] + ip)), __ldcg(P.z + ip + dip), hp);
  if (in_q) hq = fma(-(P.om * ldc<T, TC>(c[4] + iq)), __ldcg(P.z + iq + diq), hq);
  const T gab = P.om * ldc<T, TC>(c[1] + ip), gba = P.om * ldc<T, TC>(c[2] + iq);
  C.hp[j] = hp;
  C.hq[j] = hq;
  C.a[j] = k > 0 ? P.om * ldc<T, TC>(c[0] + ip) : T(0);
  C.b[j] = k > 0 ? P.om * ldc<T, TC>(c[0] + iq) : T(0);
  C.gab[j] = gab;
  C.gba[j] = gba;
  C.idet[j] = T(1) / fma(-gab, gba, T(1));
}

// Lane 0: pairs j < m of the chunk, in chain order; results replace hp / hq.
template <class T>
__device__ __forceinline__ void run_chunk(Chunk<T>& C, int m, T& zp, T& zq) {
#pragma unroll 4
  for (int j = 0; j < m; ++j) {
    const T hp = fma(-C.a[j], zp, C.hp[j]);
    const T hq = fma(-C.b[j], zq, C.hq[j]);
    zp = fma(-C.gab[j], hq, hp) * C.idet[j];
    zq = fma(-C.gba[j], hp, hq) * C.idet[j];
    C.hp[j] = zp;
    C.hq[j] = zq;
  }
}

template <class T, class TC>
__device__ __forceinline__ void edges_body(const EdgeP<T, TC>& P, int id, int lane, Chunk<T>& C) {
  const int px = P.sx.p, py = P.sy.p;
  const int ny_tasks = px * (py - 1), nx_tasks = (px - 1) * py;
  if (id >= ny_tasks + nx_tasks) return;
  int vx = -1, vy = -1;
  // chain geometry: first cell of pair k is ip(k) = i0 - k * step, second iq = ip + dq
  int64_t i0 = 0, step = 0, dq = 0, dip = 0, diq = 0;
  int npairs = 0, en = 0, eab = 0, eba = 0, eip = 0, eiq = 0;
  bool in_p = false, in_q = false;
  if (id < ny_tasks) {
    // interface between (ix, iy) below and (ix, iy+1) above; pairs along x
    const int ix = id % px, iy = id / px;
    const int c = P.base ^ (ix & 1) ^ ((iy & 1) << 1);
    if (!((c >> 1) & 1)) return;  // coupled only if both start here
    const int cx = c & 1;
    const int gx0 = P.sx.lo(ix), w = P.sx.len(ix);
    const int Y = P.sy.lo(iy) + P.sy.len(iy) - 1;
    in_p = P.sy.len(iy) >= 2;
    in_q = P.sy.len(iy + 1) >= 2;
    const int dx = cx ? -1 : 1;
    const int ge = cx ? gx0 : gx0 + w - 1;  // far end of the chain
    const bool corner = cx ? (gx0 + w < P.nx) : (gx0 > 0);
    if (corner) {
      vx = cx ? ix : ix - 1;
      vy = iy;
    }
    // the start column belongs to the corner system when there is one
    npairs = corner ? w - 1 : w;
    i0 = (int64_t)Y * P.nx + ge;
    step = dx;
    dq = P.nx;
    en = cx ? 0 : 1;  // entry towards the previous pair along the chain
    eab = 3;
    eba = 2;
    eip = 2;
    dip = -P.nx;
    eiq = 3;
    diq = P.nx;
  } else {
    // interface between (ix, iy) left and (ix+1, iy) right; pairs along y
    const int k = id - ny_tasks;
    const int ix = k % (px - 1), iy = k / (px - 1);
    const int c = P.base ^ (ix & 1) ^ ((iy & 1) << 1);
    if (!(c & 1)) return;
    const int cy = (c >> 1) & 1;
    const int gy0 = P.sy.lo(iy), h = P.sy.len(iy);
    const int X = P.sx.lo(ix) + P.sx.len(ix) - 1;
    in_p = P.sx.len(ix) >= 2;
    in_q = P.sx.len(ix + 1) >= 2;
    const int dy = cy ? -1 : 1;
    const int ge = cy ? gy0 : gy0 + h - 1;
    const bool corner = cy ? (gy0 + h < P.ny) : (gy0 > 0);
    if (corner) {
      vx = ix;
      vy = cy ? iy : iy - 1;
    }
    npairs = corner ? h - 1 : h;
    i0 = (int64_t)ge * P.nx + X;
    step = (int64_t)dy * P.nx;
    dq = 1;
    en = cy ? 2 : 3;
    eab = 1;
    eba = 0;
    eip = 0;
    dip = -1;
    eiq = 1;
    diq = 1;
  }
  const TC* const c[5] = {P.cT[en], P.cT[eab], P.cT[eba], P.cT[eip], P.cT[eiq]};
  T zp = T(0), zq = T(0);
  for (int k0 = 0; k0 < npairs; k0 += ELN) {
    const int k = k0 + lane;
    const int64_t ip = i0 - (int64_t)k * step, iq = ip + dq;
    if (k < npairs) stage_pair(P, c, C, lane, k, ip, iq, dip, diq, in_p, in_q);
    __syncwarp();
    if (lane == 0) run_chunk(C, min(ELN, npairs - k0), zp, zq);
    __syncwarp();
    if (k < npairs) {
      P.z[ip] = C.hp[lane];
      P.z[iq] = C.hq[lane];
    }
    __syncwarp();
  }
  if (vx >= 0) {
    __threadfence();  // every lane's chain values before the arrival
    __syncwarp();
    if (lane == 0) {
      const unsigned vid = (unsigned)(vx + (px - 1) * vy);
      if (atomicAdd(&P.vcount[vid], 1u) == 3u) {
        P.vcount[vid] = 0;  // ready for the next apply
        __threadfence();
        solve_vertex(P, vx, vy);
      }
    }
  }
}

template <class TC>
__global__ void transposed_set_kernel(int nx, int ny, int nz, int s, int64_t N, const double* A, TC* out) {
  const int64_t pl = (int64_t)nx * ny;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % nx), y = (int)((i / nx) % ny), z = (int)(i / pl);
    const double inv = 1.0 / A[i];
    out[i] = (TC)inv;
    // entry e of row i points to j; the transposed entry is A(j, opposite of e)
    const double w = x > 0 ? A[2 * N + i - 1] : 0.0;        // A(i-1, E)
    const double e = x + 1 < nx ? A[1 * N + i + 1] : 0.0;   // A(i+1, W)
    const double so = y > 0 ? A[4 * N + i - nx] : 0.0;      // A(i-nx, N)
    const double n = y + 1 < ny ? A[3 * N + i + nx] : 0.0;  // A(i+nx, S)
    out[1 * N + i] = (TC)(w * inv);
    out[2 * N + i] = (TC)(e * inv);
    out[3 * N + i] = (TC)(so * inv);
    out[4 * N + i] = (TC)(n * inv);
    if (s == 7) {
      const double b = z > 0 ? A[6 * N + i - pl] : 0.0;       // A(i-pl, F)
      const double f = z + 1 < nz ? A[5 * N + i + pl] : 0.0;  // A(i+pl, B)
      out[5 * N + i] = (TC)(b * inv);
      out[6 * N + i] = (TC)(f * inv);
    }
  }
}

template <class T, class TC>
__global__ void __launch_bounds__(ETH) ssor_edges_kernel(EdgeP<T, TC> P) {
  __shared__ Chunk<T> C[ECH];
  const int wid = threadIdx.x / ELN;
  edges_body(P, blockIdx.x * ECH + wid, threadIdx.x % ELN, C[wid]);
}

// The interface chains of several problems: problem p owns blocks
// off[p] .. off[p+1] - 1 (ECH chains each).
template <class T, class TC>
__global__ void __launch_bounds__(ETH) ssor_edges_batch_kernel(const EdgeP<T, TC>* __restrict__ Pa,
                                                              const unsigned* __restrict__ off, int np) {
  __shared__ Chunk<T> C[ECH];
  int lo = 0, hi = np - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= blockIdx.x) lo = mid;
    else hi = mid - 1;
  }
  const int wid = threadIdx.x / ELN;
  edges_body(Pa[lo], (int)(blockIdx.x - off[lo]) * ECH + wid, threadIdx.x % ELN, C[wid]);
}

template <class T, class TC>
ndiag_status edge_params(Handle* h, double omega, const void* w, void* z, EdgeP<T, TC>& P, int& tasks) {
  P = EdgeP<T, TC>{};
  P.nx = (int)h->n[0];
  P.ny = (int)h->n[1];
  const int px = h->sub[0], py = h->sub[1];
  P.sx = Split{px, P.nx / px, P.nx % px};
  P.sy = Split{py, P.ny / py, P.ny % py};
  P.base = base_corner(2, fwd_phase(2));
  const size_t N = (size_t)h->N;
  const TC* base = (const TC*)h->sorT.base;
  for (int e = 0; e < 4; ++e) P.cT[e] = base + (1 + e) * N;
  P.w = (const T*)w;
  P.z = (T*)z;
  P.om = (T)omega;
  tasks = px * (py - 1) + (px - 1) * py;
  if (tasks <= 0) return NDIAG_OK;
  const size_t vbytes = sizeof(unsigned) * (size_t)((px - 1) * (py - 1) + 1);
  if (h->vcount_bytes < vbytes) {
    dev_free(h->vcount, h->vcount_bytes, h->stream);
    h->vcount = (unsigned*)dev_alloc(vbytes, h->stream);
    if (!h->vcount) return NDIAG_ENOMEM;
    h->vcount_bytes = vbytes;
    ND_CUDA(cudaMemsetAsync(h->vcount, 0, vbytes, h->stream));
  }
  P.vcount = h->vcount;
  return NDIAG_OK;
}

template <class T, class TC>
ndiag_status run_edges(Handle* h, int mode, double omega, const void* w, void* z) {
  if (mode == NDIAG_NATURAL) return NDIAG_OK;  // one subdomain: no interfaces
  EdgeP<T, TC> P;
  int tasks = 0;
  ND_TRY(edge_params(h, omega, w, z, P, tasks));
  if (tasks <= 0) return NDIAG_OK;
  ++h->launches;
  ssor_edges_kernel<T, TC><<<(tasks + ECH - 1) / ECH, ETH, 0, h->stream>>>(P);
  ND_CUDA(cudaGetLastError());
  return NDIAG_OK;
}

template <class T, class TC>
ndiag_status edges_prepare_t(BatchSweep& b, Handle* const* hs, int np, double omega, const void* const* w,
                             void* const* z, cudaStream_t s) {
  std::vector<EdgeP<T, TC>> ps((size_t)np);
  std::vector<unsigned> off((size_t)np + 1, 0);
  for (int p = 0; p < np; ++p) {
    int tasks = 0;
    ND_TRY(edge_params(hs[p], omega, w[p], z[p], ps[p], tasks));
    off[p + 1] = off[p] + (unsigned)((std::max(tasks, 0) + ECH - 1) / ECH);
  }
  const size_t pb = sizeof(EdgeP<T, TC>) * (size_t)np, ob = sizeof(unsigned) * (size_t)(np + 1);
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
  b.precision = hs[0]->precision;
  return NDIAG_OK;
}

}  // namespace

ndiag_status build_scaled_transposed(Handle* h, ScaledSet& set) {
  const size_t cs = h->precision == NDIAG_FP64 ? 8 : h->precision == NDIAG_FP32 ? 4 : 2;
  const size_t bytes = cs * (size_t)h->stencil * (size_t)h->N;
  if (!set.base) {
    set.base = dev_alloc(bytes, h->stream);
    if (!set.base) return NDIAG_ENOMEM;
    set.bytes = bytes;
  }
  const int nx = (int)h->n[0], ny = (int)h->n[1], nz = (int)h->n[2];
  const int grid = h->sm_count * 4;
  ++h->launches;
  ++set.version;
  if (h->precision == NDIAG_FP64)
    transposed_set_kernel<double><<<grid, 256, 0, h->stream>>>(nx, ny, nz, h->stencil, h->N, h->A64, (double*)set.base);
  else if (h->precision == NDIAG_FP32)
    transposed_set_kernel<float><<<grid, 256, 0, h->stream>>>(nx, ny, nz, h->stencil, h->N, h->A64, (float*)set.base);
  else
    transposed_set_kernel<__half><<<grid, 256, 0, h->stream>>>(nx, ny, nz, h->stencil, h->N, h->A64, (__half*)set.base);
  ND_CUDA(cudaGetLastError());
  return NDIAG_OK;
}

ndiag_status batch_edges_prepare(BatchSweep& b, Handle* const* hs, int np, double omega, const void* const* w,
                                 void* const* z, cudaStream_t s) {
  if (np < 1) return NDIAG_EINVAL;
  switch (hs[0]->precision) {
    case NDIAG_FP64: return edges_prepare_t<double, double>(b, hs, np, omega, w, z, s);
    case NDIAG_FP32: return edges_prepare_t<float, float>(b, hs, np, omega, w, z, s);
  }
  return NDIAG_EINVAL;
}

ndiag_status batch_edges_launch(const BatchSweep& b, cudaStream_t s) {
  if (b.total == 0) return NDIAG_OK;
  if (b.precision == NDIAG_FP64)
    ssor_edges_batch_kernel<double, double><<<b.total, ETH, 0, s>>>((const EdgeP<double, double>*)b.params, b.off,
                                                                     b.np);
  else
    ssor_edges_batch_kernel<float, float><<<b.total, ETH, 0, s>>>((const EdgeP<float, float>*)b.params, b.off, b.np);
  ND_CUDA(cudaGetLastError());
  return NDIAG_OK;
}

ndiag_status launch_ssor_edges2d(Handle* h, int mode, double omega, const void* w, void* z) {
  switch (h->precision) {
    case NDIAG_FP64: return run_edges<double, double>(h, mode, omega, w, z);
    case NDIAG_FP32: return run_edges<float, float>(h, mode, omega, w, z);
    default: return run_edges<float, __half>(h, mode, omega, w, z);
  }
}

}  // namespace nd
