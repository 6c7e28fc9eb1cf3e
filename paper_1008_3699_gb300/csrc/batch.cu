// Batched solves of many independent 2D 5-point problems of different sizes
// (one handle per problem): FP32 SSOR-preconditioned CG inner solves (the
// paper's decomposed SSOR, Sec. 5) wrapped in FP64 iterative refinement.
//
// Every step of an iteration is ONE launch over all problems: the sweeps of
// the SSOR apply run through the staged sweep kernel with a per-problem
// parameter array, vector operations walk a block table (each block a run of
// cells of one problem), and dot products are summed per problem in block
// order (deterministic, so a problem's arithmetic does not depend on the
// others in the batch). Per-problem scalars and convergence masks stay on the
// device. The inner iterations of a refinement step are one launch of a CUDA
// graph whose conditional while node repeats a captured body of 8 iterations
// until no problem is active (the device sets the condition); a converged
// problem keeps its slot (alpha = 0), so the body is static.
//
// The subdomain partition ("tile") of every problem is chosen by an
// autotuner: for each candidate tile side it times batched SSOR applies and
// counts the iterations of pilot solves, and keeps the cheapest product.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.h"

namespace nd {
namespace {

constexpr int VB = 1024;  // cells per block of the vector kernels
constexpr int VT = 256;   // threads per block

struct BProb {
  int nx, ny;
  int64_t off;  // first cell in the concatenated vectors
  const double* A64;
  const float* A32;
};

__device__ __forceinline__ double stencil64(const BProb& p, const double* x, int64_t i) {
  const int64_t N = (int64_t)p.nx * p.ny;
  const int cx = (int)(i % p.nx), cy = (int)(i / p.nx);
  double acc = p.A64[i] * x[i];
  if (cx > 0) acc = fma(p.A64[N + i], x[i - 1], acc);
  if (cx + 1 < p.nx) acc = fma(p.A64[2 * N + i], x[i + 1], acc);
  if (cy > 0) acc = fma(p.A64[3 * N + i], x[i - p.nx], acc);
  if (cy + 1 < p.ny) acc = fma(p.A64[4 * N + i], x[i + p.nx], acc);
  return acc;
}
__device__ __forceinline__ float stencil32(const BProb& p, const float* x, int64_t i) {
  const int64_t N = (int64_t)p.nx * p.ny;
  const int cx = (int)(i % p.nx), cy = (int)(i / p.nx);
  float acc = p.A32[i] * x[i];
  if (cx > 0) acc = fmaf(p.A32[N + i], x[i - 1], acc);
  if (cx + 1 < p.nx) acc = fmaf(p.A32[2 * N + i], x[i + 1], acc);
  if (cy > 0) acc = fmaf(p.A32[3 * N + i], x[i - p.nx], acc);
  if (cy + 1 < p.ny) acc = fmaf(p.A32[4 * N + i], x[i + p.nx], acc);
  return acc;
}

// block sum of one double per thread into part[blockIdx.x * stride + k]
__device__ __forceinline__ void block_sum(double v, double* out) {
  __shared__ double sh[VT / 32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = threadIdx.x < VT / 32 ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) *out = v;
  }
  __syncthreads();
}

struct Blocks {
  const int* pid;
  const int64_t* start;  // cell within the problem
  const BProb* prob;
};

#define BLOCK_RANGE                                     \
  const int pid = B.pid[blockIdx.x];                    \
  const BProb P = B.prob[pid];                          \
  const int64_t c0 = B.start[blockIdx.x];               \
  const int64_t N = (int64_t)P.nx * P.ny;               \
  const int64_t c1 = c0 + VB < N ? c0 + VB : N;

// r = b - A x (fp64), part = (r, r); r32 = (float) r when outer-active else 0
__global__ void __launch_bounds__(VT) k_resid(Blocks B, const double* b, const double* x, double* r, float* r32,
                                              const int* oact, double* part) {
  BLOCK_RANGE
  double s = 0.0;
  for (int64_t c = c0 + threadIdx.x; c < c1; c += VT) {
    const int64_t g = P.off + c;
    const double v = b[g] - stencil64(P, x + P.off, c);
    r[g] = v;
    r32[g] = oact[pid] ? (float)v : 0.0f;
    s = fma(v, v, s);
  }
  block_sum(s, part + blockIdx.x);
}

// part = (x, y)
__global__ void __launch_bounds__(VT) k_dot(Blocks B, const float* x, const float* y, double* part) {
  BLOCK_RANGE
  double s = 0.0;
  for (int64_t c = c0 + threadIdx.x; c < c1; c += VT) {
    const int64_t g = P.off + c;
    s = fma((double)x[g], (double)y[g], s);
  }
  block_sum(s, part + blockIdx.x);
}

// q = A p, part = (p, q)
__global__ void __launch_bounds__(VT) k_spmv_dot(Blocks B, const float* p, float* q, double* part) {
  BLOCK_RANGE
  double s = 0.0;
  for (int64_t c = c0 + threadIdx.x; c < c1; c += VT) {
    const int64_t g = P.off + c;
    const float v = stencil32(P, p + P.off, c);
    q[g] = v;
    s = fma((double)p[g], (double)v, s);
  }
  block_sum(s, part + blockIdx.x);
}

// e += alpha p, r -= alpha q, part = (r, r)
__global__ void __launch_bounds__(VT) k_update(Blocks B, const double* alpha, float* e, const float* p, float* r,
                                               const float* q, double* part) {
  BLOCK_RANGE
  const float a = (float)alpha[pid];
  double s = 0.0;
  for (int64_t c = c0 + threadIdx.x; c < c1; c += VT) {
    const int64_t g = P.off + c;
    e[g] = fmaf(a, p[g], e[g]);
    const float rv = fmaf(-a, q[g], r[g]);
    r[g] = rv;
    s = fma((double)rv, (double)rv, s);
  }
  block_sum(s, part + blockIdx.x);
}

// part = (x, x) in fp64
__global__ void __launch_bounds__(VT) k_dot64(Blocks B, const double* x, double* part) {
  BLOCK_RANGE
  double s = 0.0;
  for (int64_t c = c0 + threadIdx.x; c < c1; c += VT) s = fma(x[P.off + c], x[P.off + c], s);
  block_sum(s, part + blockIdx.x);
}

// p = z + beta p (first: p = z)
__global__ void __launch_bounds__(VT) k_pupd(Blocks B, const double* beta, const float* z, float* p, int first) {
  BLOCK_RANGE
  const float bt = first ? 0.0f : (float)beta[pid];
  for (int64_t c = c0 + threadIdx.x; c < c1; c += VT) {
    const int64_t g = P.off + c;
    p[g] = first ? z[g] : fmaf(bt, p[g], z[g]);
  }
}

// x += e (outer-active problems), e = 0
__global__ void __launch_bounds__(VT) k_correct(Blocks B, double* x, float* e, const int* oact) {
  BLOCK_RANGE
  const bool on = oact[pid] != 0;
  for (int64_t c = c0 + threadIdx.x; c < c1; c += VT) {
    const int64_t g = P.off + c;
    if (on) x[g] += (double)e[g];
    e[g] = 0.0f;
  }
}

__global__ void k_zero32(float* v, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    v[i] = 0.0f;
}

// per-problem sum of its blocks' partials, in block order
__global__ void k_reduce(int np, const int* blk0, const double* part, double* out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  double s = 0.0;
  for (int k = blk0[p]; k < blk0[p + 1]; ++k) s += part[k];
  out[p] = s;
}

struct Scal {
  double *rz, *rr, *r0r0, *pq, *alpha, *beta, *bb, *rr64, *tmp;
  int *act, *oact, *iters, *outer, *nact;
  int *inner, *maxit;  // iterations of the current inner loop, and its limit
};

// inner start: rz = (r, z) (in tmp); the inner stop threshold on (r, r):
// t^2 (r0, r0) with t = 0.5 rtol ||b|| / ||r_outer|| clamped to [1e-6, 1e-3]
// (one inner solve aims at the outer tolerance; fp32 gains nothing below
// 1e-6); active = outer-active and (r0, r0) > 0
__global__ void k_inner_init(int np, Scal s, double rtol) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  s.rz[p] = s.tmp[p];
  const double rn = sqrt(s.rr64[p]);
  double t = rn > 0.0 ? 0.5 * rtol * sqrt(s.bb[p]) / rn : 1e-3;
  t = fmin(1e-3, fmax(1e-6, t));
  s.r0r0[p] = s.rr[p] * t * t;
  s.act[p] = s.oact[p] && s.rr[p] > 0.0;
}
__global__ void k_alpha(int np, Scal s) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  const bool on = s.act[p] && s.pq[p] != 0.0 && s.rz[p] != 0.0;
  s.alpha[p] = on ? s.rz[p] / s.pq[p] : 0.0;
  if (!on) s.act[p] = 0;
}
// after the update: inner convergence on the recurrence residual
__global__ void k_check(int np, Scal s, double tol2) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  if (s.act[p]) {
    s.iters[p] += 1;
    if (s.rr[p] <= tol2 * s.r0r0[p]) s.act[p] = 0;  // r0r0 holds the threshold (tol2 = 1)
  }
}
// beta = (r, z)_new / (r, z)
__global__ void k_beta(int np, Scal s) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  const double rzn = s.tmp[p];
  s.beta[p] = (s.act[p] && s.rz[p] != 0.0) ? rzn / s.rz[p] : 0.0;
  s.rz[p] = rzn;
}
__global__ void k_count(int np, const int* a, int* n) {
  __shared__ int cnt;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  int c = 0;
  for (int p = threadIdx.x; p < np; p += blockDim.x) c += a[p] != 0;
  atomicAdd(&cnt, c);
  __syncthreads();
  if (threadIdx.x == 0) *n = cnt;
}
// outer step: relres = sqrt(rr64 / bb); outer-active = relres > rtol
// End of a body of the inner while-loop (k iterations): the loop goes on
// while some problem's inner iteration is active and the limit is not reached.
__global__ void k_inner_cond(int np, Scal s, int k, cudaGraphConditionalHandle cond) {
  int mine = 0;
  for (int p = threadIdx.x; p < np; p += blockDim.x) mine |= s.act[p];
  const int any = __syncthreads_or(mine);
  if (threadIdx.x == 0) {
    const int n = *s.inner + k;
    *s.inner = n;
    cudaGraphSetConditional(cond, (any && n < *s.maxit) ? 1u : 0u);
  }
}

__global__ void k_outer(int np, Scal s, double rtol) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  const double rel = s.bb[p] > 0.0 ? sqrt(s.rr64[p] / s.bb[p]) : 0.0;
  const int was = s.oact[p];
  s.oact[p] = rel > rtol;
  if (was && s.oact[p]) s.outer[p] += 1;
}

}  // namespace

// Re-partition a handle (the autotuner): drops what depends on the partition.
void handle_set_sub(Handle* h, const int sub[3]) {
  for (LineTable& t : h->line_tables) dev_free(t.buf, t.bytes, h->stream);
  h->line_tables.clear();
  for (int a = 0; a < 3; ++a) h->sub[a] = a < h->dim ? std::max(1, std::min<int>(sub[a], (int)h->n[a])) : 1;
  dev_free(h->vcount, h->vcount_bytes, h->stream);
  h->vcount = nullptr;
  h->vcount_bytes = 0;
}

}  // namespace nd

using namespace nd;

struct ndiag_batch {
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int np = 0;
  std::vector<ndiag*> hs;
  std::vector<int> tile;  // chosen tile side per problem
  std::vector<int64_t> off;
  int64_t Ntot = 0;
  BProb* prob = nullptr;
  int nblk = 0;
  int* blk_pid = nullptr;
  int64_t* blk_start = nullptr;
  int* blk0 = nullptr;
  double *b64 = nullptr, *x64 = nullptr, *r64 = nullptr, *part = nullptr;
  float *r32 = nullptr, *e32 = nullptr, *p32 = nullptr, *q32 = nullptr, *z32 = nullptr, *t32 = nullptr;
  Scal sc{};
  void* scal_mem = nullptr;
  size_t scal_bytes = 0;
  int* nact_host = nullptr;
  double omega = 1.0;
  BatchSweep fwd, rev, edges;
  cudaGraphExec_t loop = nullptr;  // the inner PCG loop: one conditional while node
  std::vector<void*> allocs;
  std::vector<size_t> alloc_bytes;
  int64_t launches = 0;
};

namespace {

void* balloc(ndiag_batch* B, size_t bytes) {
  void* p = dev_alloc(bytes, B->stream);
  if (p) {
    B->allocs.push_back(p);
    B->alloc_bytes.push_back(bytes);
  }
  return p;
}

Blocks blocks(ndiag_batch* B) { return Blocks{B->blk_pid, B->blk_start, B->prob}; }

ndiag_status reduce(ndiag_batch* B, double* out) {
  k_reduce<<<(B->np + 127) / 128, 128, 0, B->stream>>>(B->np, B->blk0, B->part, out);
  ++B->launches;
  ND_CUDA(cudaGetLastError());
  return NDIAG_OK;
}

// z = M^-1 r for every problem: forward sweep, reversed interior, interface chains
ndiag_status ssor_batch(ndiag_batch* B) {
  ND_TRY(batch_sweep_launch(B->fwd, B->stream));
  ND_TRY(batch_sweep_launch(B->rev, B->stream));
  ND_TRY(batch_edges_launch(B->edges, B->stream));
  B->launches += 3;
  return NDIAG_OK;
}

ndiag_status prepare_sweeps(ndiag_batch* B) {
  const int np = B->np;
  std::vector<const void*> r(np), t(np);
  std::vector<void*> tw(np), z(np);
  for (int p = 0; p < np; ++p) {
    r[p] = B->r32 + B->off[p];
    t[p] = B->t32 + B->off[p];
    tw[p] = B->t32 + B->off[p];
    z[p] = B->z32 + B->off[p];
    if (!B->hs[p]->sorT.base) ND_TRY(build_scaled_transposed(B->hs[p], B->hs[p]->sorT));
  }
  const double w = B->omega;
  const double om[8] = {w, w, w, w, w, w, w, w};
  const int64_t tf = fwd_phase(2);
  std::vector<Handle*> hh(B->hs.begin(), B->hs.end());
  ND_TRY(batch_sweep_prepare(B->fwd, hh.data(), np, KIND_TRI_SCALED, NDIAG_DECOMPOSED, tf, om, 0, r.data(), nullptr,
                             tw.data(), w * (2.0 - w), false, B->stream));
  ND_TRY(batch_sweep_prepare(B->rev, hh.data(), np, KIND_TRI_UNIT, NDIAG_DECOMPOSED, tf ^ 1, om, 2, t.data(), nullptr,
                             z.data(), 1.0, true, B->stream));
  ND_TRY(batch_edges_prepare(B->edges, hh.data(), np, w, t.data(), z.data(), B->stream));
  if (B->loop) {
    cudaGraphExecDestroy(B->loop);
    B->loop = nullptr;
  }
  return NDIAG_OK;
}

// One inner PCG iteration for all problems (capturable).
ndiag_status pcg_iteration(ndiag_batch* B, double tol2) {
  const Blocks bl = blocks(B);
  const int g = B->nblk, np = B->np, pg = (np + 127) / 128;
  k_spmv_dot<<<g, VT, 0, B->stream>>>(bl, B->p32, B->q32, B->part);
  ND_TRY(reduce(B, B->sc.pq));
  k_alpha<<<pg, 128, 0, B->stream>>>(np, B->sc);
  k_update<<<g, VT, 0, B->stream>>>(bl, B->sc.alpha, B->e32, B->p32, B->r32, B->q32, B->part);
  ND_TRY(reduce(B, B->sc.rr));
  k_check<<<pg, 128, 0, B->stream>>>(np, B->sc, tol2);
  ND_TRY(ssor_batch(B));
  k_dot<<<g, VT, 0, B->stream>>>(bl, B->r32, B->z32, B->part);
  ND_TRY(reduce(B, B->sc.tmp));
  k_beta<<<pg, 128, 0, B->stream>>>(np, B->sc);
  k_pupd<<<g, VT, 0, B->stream>>>(bl, B->sc.beta, B->z32, B->p32, 0);
  B->launches += 6;
  ND_CUDA(cudaGetLastError());
  return NDIAG_OK;
}

ndiag_status count_active(ndiag_batch* B, const int* flags, int* n) {
  k_count<<<1, 256, 0, B->stream>>>(B->np, flags, B->sc.nact);
  ND_CUDA(cudaMemcpyAsync(B->nact_host, B->sc.nact, sizeof(int), cudaMemcpyDeviceToHost, B->stream));
  ND_CUDA(cudaStreamSynchronize(B->stream));
  *n = *B->nact_host;
  return NDIAG_OK;
}

// The inner PCG iterations as one executable graph: a conditional while node
// whose body holds K iterations (every step one launch over all problems) and
// the condition kernel. The body is captured from the stream.
constexpr int LOOP_K = 8;
ndiag_status build_loop(ndiag_batch* B) {
  cudaGraph_t g = nullptr;
  ND_CUDA(cudaGraphCreate(&g, 0));
  cudaGraphConditionalHandle cond;
  cudaError_t e = cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault);
  cudaGraphNodeParams np{};
  cudaGraphNode_t node;
  if (e == cudaSuccess) {
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = cond;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np);
  }
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return cuda_status(e, "conditional while node");
  }
  cudaGraph_t body = np.conditional.phGraph_out[0];
  e = cudaStreamBeginCaptureToGraph(B->stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return cuda_status(e, "cudaStreamBeginCaptureToGraph(inner loop)");
  }
  const int64_t l0 = B->launches;
  ndiag_status st = NDIAG_OK;
  for (int k = 0; k < LOOP_K && st == NDIAG_OK; ++k) st = pcg_iteration(B, 1.0);
  if (st == NDIAG_OK) {
    k_inner_cond<<<1, 256, 0, B->stream>>>(B->np, B->sc, LOOP_K, cond);
    e = cudaGetLastError();
  }
  cudaGraph_t got = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(B->stream, &got);
  B->launches = l0;  // captured, not run
  if (st == NDIAG_OK && e == cudaSuccess && e2 == cudaSuccess) e = cudaGraphInstantiate(&B->loop, g, 0);
  cudaGraphDestroy(g);
  if (st != NDIAG_OK) return st;
  if (e != cudaSuccess || e2 != cudaSuccess) {
    B->loop = nullptr;
    return cuda_status(e != cudaSuccess ? e : e2, "inner loop graph");
  }
  return NDIAG_OK;
}

// Batched solve of every problem: x (device, concatenated) in/out.
ndiag_status batch_solve(ndiag_batch* B, const double* b, double* x, double rtol, int maxit,
                         std::vector<int>& iters, std::vector<int>& outer, std::vector<double>& relres) {
  const Blocks bl = blocks(B);
  const int g = B->nblk, np = B->np, pg = (np + 127) / 128;
  {
    const int lim = std::max(maxit, 1);
    ND_CUDA(cudaMemcpyAsync(B->sc.maxit, &lim, sizeof(int), cudaMemcpyHostToDevice, B->stream));
  }
  // ||b||^2 per problem
  ND_CUDA(cudaMemcpyAsync(B->b64, b, sizeof(double) * B->Ntot, cudaMemcpyDeviceToDevice, B->stream));
  ND_CUDA(cudaMemcpyAsync(B->x64, x, sizeof(double) * B->Ntot, cudaMemcpyDeviceToDevice, B->stream));
  ND_CUDA(cudaMemsetAsync(B->sc.iters, 0, sizeof(int) * np, B->stream));
  ND_CUDA(cudaMemsetAsync(B->sc.outer, 0, sizeof(int) * np, B->stream));
  {
    std::vector<int> ones(np, 1);
    ND_CUDA(cudaMemcpyAsync(B->sc.oact, ones.data(), sizeof(int) * np, cudaMemcpyHostToDevice, B->stream));
    ND_CUDA(cudaStreamSynchronize(B->stream));
  }
  k_dot64<<<g, VT, 0, B->stream>>>(bl, B->b64, B->part);
  ND_TRY(reduce(B, B->sc.bb));
  int nouter = 0;
  for (;;) {
    // true fp64 residual, outer-active update, fp32 inner right-hand side
    k_resid<<<g, VT, 0, B->stream>>>(bl, B->b64, B->x64, B->r64, B->r32, B->sc.oact, B->part);
    ND_TRY(reduce(B, B->sc.rr64));
    k_outer<<<pg, 128, 0, B->stream>>>(np, B->sc, rtol);
    // r32 was filled with the previous outer-active mask; clear converged ones
    k_resid<<<g, VT, 0, B->stream>>>(bl, B->b64, B->x64, B->r64, B->r32, B->sc.oact, B->part);
    int nact = 0;
    ND_TRY(count_active(B, B->sc.oact, &nact));
    if (nact == 0 || nouter >= 60) break;
    ++nouter;
    // inner PCG start
    k_zero32<<<1024, 256, 0, B->stream>>>(B->e32, B->Ntot);
    ND_TRY(ssor_batch(B));
    k_dot<<<g, VT, 0, B->stream>>>(bl, B->r32, B->z32, B->part);
    ND_TRY(reduce(B, B->sc.tmp));
    k_dot<<<g, VT, 0, B->stream>>>(bl, B->r32, B->r32, B->part);
    ND_TRY(reduce(B, B->sc.rr));
    k_inner_init<<<pg, 128, 0, B->stream>>>(np, B->sc, rtol);
    k_pupd<<<g, VT, 0, B->stream>>>(bl, B->sc.beta, B->z32, B->p32, 1);
    ND_CUDA(cudaGetLastError());
    // the inner iterations: one launch of the while-loop graph (the device
    // decides when they stop)
    if (!B->loop) ND_TRY(build_loop(B));
    ND_CUDA(cudaMemsetAsync(B->sc.inner, 0, sizeof(int), B->stream));
    ND_CUDA(cudaGraphLaunch(B->loop, B->stream));
    ++B->launches;
    k_correct<<<g, VT, 0, B->stream>>>(bl, B->x64, B->e32, B->sc.oact);
    ND_CUDA(cudaGetLastError());
  }
  ND_CUDA(cudaMemcpyAsync(x, B->x64, sizeof(double) * B->Ntot, cudaMemcpyDeviceToDevice, B->stream));
  std::vector<double> rr(np), bb(np);
  iters.assign(np, 0);
  outer.assign(np, 0);
  relres.assign(np, 0.0);
  ND_CUDA(cudaMemcpyAsync(iters.data(), B->sc.iters, sizeof(int) * np, cudaMemcpyDeviceToHost, B->stream));
  ND_CUDA(cudaMemcpyAsync(outer.data(), B->sc.outer, sizeof(int) * np, cudaMemcpyDeviceToHost, B->stream));
  ND_CUDA(cudaMemcpyAsync(rr.data(), B->sc.rr64, sizeof(double) * np, cudaMemcpyDeviceToHost, B->stream));
  ND_CUDA(cudaMemcpyAsync(bb.data(), B->sc.bb, sizeof(double) * np, cudaMemcpyDeviceToHost, B->stream));
  ND_CUDA(cudaStreamSynchronize(B->stream));
  // outer[p] counts the checks after which problem p stayed active, i.e. its
  // refinement steps (inner solves), as ndiag_solve_info.outer of krylov_solve
  for (int p = 0; p < np; ++p) relres[p] = bb[p] > 0 ? std::sqrt(rr[p] / bb[p]) : 0.0;
  for (ndiag* h : B->hs) ND_TRY(check_device_status(h));
  return NDIAG_OK;
}

void set_tiles(ndiag_batch* B, const std::vector<int>& tile) {
  B->tile = tile;
  for (int p = 0; p < B->np; ++p) {
    Handle* h = B->hs[p];
    const int sub[3] = {(int)((h->n[0] + tile[p] - 1) / tile[p]), (int)((h->n[1] + tile[p] - 1) / tile[p]), 1};
    handle_set_sub(h, sub);
  }
}

// Autotuner: candidate tile sides; cost = time of a batched SSOR apply x mean
// iterations of pilot single-problem solves (smallest, median, largest).
ndiag_status autotune(ndiag_batch* B) {
  const int cands[3] = {32, 64, 128};
  std::vector<int> order(B->np);
  for (int p = 0; p < B->np; ++p) order[p] = p;
  std::sort(order.begin(), order.end(), [&](int a, int b) { return B->hs[a]->N < B->hs[b]->N; });
  const int pilots[3] = {order[0], order[B->np / 2], order[B->np - 1]};
  double best = 1e300;
  int best_t = 64;
  cudaEvent_t e0, e1;
  ND_CUDA(cudaEventCreate(&e0));
  ND_CUDA(cudaEventCreate(&e1));
  for (int ci = 0; ci < 3; ++ci) {
    std::vector<int> tile(B->np, cands[ci]);
    set_tiles(B, tile);
    ND_TRY(prepare_sweeps(B));
    ND_TRY(ssor_batch(B));  // warm-up (builds line tables)
    ND_CUDA(cudaEventRecord(e0, B->stream));
    for (int k = 0; k < 3; ++k) ND_TRY(ssor_batch(B));
    ND_CUDA(cudaEventRecord(e1, B->stream));
    ND_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    ND_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    double its = 0.0;
    for (int q = 0; q < 3; ++q) {
      ndiag* h = B->hs[pilots[q]];
      const int64_t N = h->N;
      double* bx = (double*)dev_alloc(sizeof(double) * 2 * N, B->stream);
      if (!bx) return NDIAG_ENOMEM;
      ND_CUDA(cudaMemcpyAsync(bx, B->b64 + B->off[pilots[q]], sizeof(double) * N, cudaMemcpyDeviceToDevice,
                              B->stream));
      ND_CUDA(cudaMemsetAsync(bx + N, 0, sizeof(double) * N, B->stream));
      ndiag_solve_info info{};
      const double om[8] = {B->omega, B->omega, B->omega, B->omega, B->omega, B->omega, B->omega, B->omega};
      krylov_solve(h, NDIAG_PCG, NDIAG_PREC_SSOR, NDIAG_DECOMPOSED, om, 1e-8, 20000, bx, bx + N, &info);
      dev_free(bx, sizeof(double) * 2 * N, B->stream);
      its += info.iterations;
    }
    const double cost = ms / 3.0 * its;
    if (cost < best) {
      best = cost;
      best_t = cands[ci];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  std::vector<int> tile(B->np, best_t);
  set_tiles(B, tile);
  return prepare_sweeps(B);
}

}  // namespace

extern "C" {

ndiag_status ndiag_batch_create(ndiag_batch** out, int count, const int64_t* nx, const int64_t* ny,
                                const double* const* diags, const int* tile, double omega, void* stream) {
  if (!out) return NDIAG_EINVAL;
  *out = nullptr;
  if (count < 1 || !nx || !ny || !diags || !(omega > 0.0 && omega < 2.0)) return NDIAG_EINVAL;
  ndiag_batch* B = new ndiag_batch();
  B->np = count;
  B->omega = omega;
  if (stream) {
    B->stream = (cudaStream_t)stream;
  } else if (cudaStreamCreateWithFlags(&B->stream, cudaStreamNonBlocking) != cudaSuccess) {
    delete B;
    return NDIAG_EDEVICE;
  } else {
    B->own_stream = true;
  }
  ndiag_status st = NDIAG_OK;
  B->off.assign(count + 1, 0);
  for (int p = 0; p < count && st == NDIAG_OK; ++p) {
    const int64_t n[3] = {nx[p], ny[p], 1};
    const int t = tile ? std::max(1, tile[p]) : 64;
    const int sub[3] = {(int)((nx[p] + t - 1) / t), (int)((ny[p] + t - 1) / t), 1};
    ndiag* h = nullptr;
    st = ndiag_create(&h, 2, n, 5, diags[p], sub, NDIAG_FP32, B->stream);
    if (st == NDIAG_OK) {
      B->hs.push_back(h);
      B->off[p + 1] = B->off[p] + nx[p] * ny[p];
    }
  }
  if (st != NDIAG_OK) {
    ndiag_batch_destroy(B);
    return st;
  }
  B->Ntot = B->off[count];
  // problem descriptors and the block table
  std::vector<BProb> pr(count);
  std::vector<int> bp, b0(count + 1, 0);
  std::vector<int64_t> bs;
  for (int p = 0; p < count; ++p) {
    Handle* h = B->hs[p];
    pr[p] = BProb{(int)h->n[0], (int)h->n[1], B->off[p], h->A64, (const float*)h->Alo};
    b0[p] = (int)bp.size();
    for (int64_t c = 0; c < h->N; c += VB) {
      bp.push_back(p);
      bs.push_back(c);
    }
  }
  b0[count] = (int)bp.size();
  B->nblk = (int)bp.size();
  const int64_t Nt = B->Ntot;
  B->prob = (BProb*)balloc(B, sizeof(BProb) * count);
  B->blk_pid = (int*)balloc(B, sizeof(int) * B->nblk);
  B->blk_start = (int64_t*)balloc(B, sizeof(int64_t) * B->nblk);
  B->blk0 = (int*)balloc(B, sizeof(int) * (count + 1));
  B->part = (double*)balloc(B, sizeof(double) * B->nblk);
  B->b64 = (double*)balloc(B, sizeof(double) * Nt);
  B->x64 = (double*)balloc(B, sizeof(double) * Nt);
  B->r64 = (double*)balloc(B, sizeof(double) * Nt);
  float** f32s[6] = {&B->r32, &B->e32, &B->p32, &B->q32, &B->z32, &B->t32};
  for (float** f : f32s) *f = (float*)balloc(B, sizeof(float) * Nt);
  B->scal_bytes = sizeof(double) * 9 * count + sizeof(int) * (5 * count + 3);
  B->scal_mem = balloc(B, B->scal_bytes);
  cudaMallocHost(&B->nact_host, sizeof(int));
  bool ok = B->prob && B->blk_pid && B->blk_start && B->blk0 && B->part && B->b64 && B->x64 && B->r64 &&
            B->scal_mem && B->nact_host;
  for (float** f : f32s) ok = ok && *f;
  if (!ok) {
    ndiag_batch_destroy(B);
    return NDIAG_ENOMEM;
  }
  double* d = (double*)B->scal_mem;
  Scal& s = B->sc;
  s.rz = d;
  s.rr = d + count;
  s.r0r0 = d + 2 * count;
  s.pq = d + 3 * count;
  s.alpha = d + 4 * count;
  s.beta = d + 5 * count;
  s.bb = d + 6 * count;
  s.rr64 = d + 7 * count;
  s.tmp = d + 8 * count;
  int* iv = (int*)(d + 9 * count);
  s.act = iv;
  s.oact = iv + count;
  s.iters = iv + 2 * count;
  s.outer = iv + 3 * count;
  s.nact = iv + 4 * count;
  s.inner = iv + 4 * count + 1;
  s.maxit = iv + 4 * count + 2;
  cudaMemcpyAsync(B->prob, pr.data(), sizeof(BProb) * count, cudaMemcpyHostToDevice, B->stream);
  cudaMemcpyAsync(B->blk_pid, bp.data(), sizeof(int) * B->nblk, cudaMemcpyHostToDevice, B->stream);
  cudaMemcpyAsync(B->blk_start, bs.data(), sizeof(int64_t) * B->nblk, cudaMemcpyHostToDevice, B->stream);
  cudaMemcpyAsync(B->blk0, b0.data(), sizeof(int) * (count + 1), cudaMemcpyHostToDevice, B->stream);
  cudaMemsetAsync(B->scal_mem, 0, B->scal_bytes, B->stream);
  cudaMemsetAsync(B->r32, 0, sizeof(float) * Nt, B->stream);
  cudaMemsetAsync(B->b64, 0, sizeof(double) * Nt, B->stream);
  if (cudaStreamSynchronize(B->stream) != cudaSuccess) {
    ndiag_batch_destroy(B);
    return NDIAG_EDEVICE;
  }
  std::vector<int> tl(count);
  for (int p = 0; p < count; ++p) tl[p] = tile ? std::max(1, tile[p]) : 64;
  set_tiles(B, tl);
  st = prepare_sweeps(B);
  if (st != NDIAG_OK) {
    ndiag_batch_destroy(B);
    return st;
  }
  *out = B;
  return NDIAG_OK;
}

ndiag_status ndiag_batch_autotune(ndiag_batch* B, const double* b) {
  if (!B || !b) return NDIAG_EINVAL;
  ND_CUDA(cudaMemcpyAsync(B->b64, b, sizeof(double) * B->Ntot, cudaMemcpyDeviceToDevice, B->stream));
  return autotune(B);
}

ndiag_status ndiag_batch_tiles(const ndiag_batch* B, int* tile) {
  if (!B || !tile) return NDIAG_EINVAL;
  for (int p = 0; p < B->np; ++p) tile[p] = B->tile[p];
  return NDIAG_OK;
}

ndiag_status ndiag_batch_solve(ndiag_batch* B, double rtol, int maxit, const double* b, double* x,
                               ndiag_solve_info* infos) {
  if (!B || !b || !x || !(rtol > 0.0) || maxit < 1) return NDIAG_EINVAL;
  const auto t0 = std::chrono::steady_clock::now();
  std::vector<int> it, ou;
  std::vector<double> rel;
  ndiag_status st = batch_solve(B, b, x, rtol, maxit, it, ou, rel);
  const double sec = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (infos) {
    for (int p = 0; p < B->np; ++p) {
      infos[p].iterations = p < (int)it.size() ? it[p] : 0;
      infos[p].outer = p < (int)ou.size() ? ou[p] : 0;
      infos[p].relres = p < (int)rel.size() ? rel[p] : 0.0;
      infos[p].seconds = sec;
      infos[p].status = st != NDIAG_OK ? st : (infos[p].relres <= rtol ? NDIAG_OK : NDIAG_ENOCONV);
    }
  }
  if (st == NDIAG_OK)
    for (int p = 0; p < B->np; ++p)
      if (rel[p] > rtol) return NDIAG_ENOCONV;
  return st;
}

int64_t ndiag_batch_cells(const ndiag_batch* B) { return B ? B->Ntot : 0; }
int64_t ndiag_batch_launches(const ndiag_batch* B) { return B ? B->launches : 0; }

// One batched SSOR apply (the preconditioner of the batched PCG) on caller
// vectors: z = M^-1 r for every problem, through the solver's own buffers.
ndiag_status ndiag_batch_ssor_apply(ndiag_batch* B, const float* r, float* z) {
  if (!B || !r || !z) return NDIAG_EINVAL;
  const size_t bytes = sizeof(float) * (size_t)B->Ntot;
  ND_CUDA(cudaMemcpyAsync(B->r32, r, bytes, cudaMemcpyDeviceToDevice, B->stream));
  ND_TRY(ssor_batch(B));
  ND_CUDA(cudaMemcpyAsync(z, B->z32, bytes, cudaMemcpyDeviceToDevice, B->stream));
  ND_CUDA(cudaStreamSynchronize(B->stream));
  for (ndiag* h : B->hs) ND_TRY(check_device_status(h));
  return NDIAG_OK;
}

void ndiag_batch_destroy(ndiag_batch* B) {
  if (!B) return;
  if (B->loop) cudaGraphExecDestroy(B->loop);
  batch_sweep_free(B->fwd, B->stream);
  batch_sweep_free(B->rev, B->stream);
  batch_sweep_free(B->edges, B->stream);
  for (size_t k = 0; k < B->allocs.size(); ++k) dev_free(B->allocs[k], B->alloc_bytes[k], B->stream);
  for (ndiag* h : B->hs) ndiag_destroy(h);
  if (B->nact_host) cudaFreeHost(B->nact_host);
  cudaStreamSynchronize(B->stream);
  if (B->own_stream) cudaStreamDestroy(B->stream);
  delete B;
}

}  // extern "C"
