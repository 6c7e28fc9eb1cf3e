// Krylov drivers: PCG, right-preconditioned BiCGSTAB, the stationary SOR
// iteration, and fp64 iterative refinement around fp32 inner solves. Scalars
// stay on the device; the host reads the residual norms once or twice per
// iteration to decide convergence.
#include <algorithm>
#include <chrono>
#include <cmath>

#include "blas.h"
#include "internal.h"

namespace nd {

ndiag_status do_ilu_apply(Handle* h, const void* r, void* z);
ndiag_status do_ilu_apply_pre(Handle* h, const void* rs, void* z);
bool ilu_prescaled_ok(const Handle* h);
const double* ilu_pivot_inverse(const Handle* h);
ndiag_status do_ssor_apply(Handle* h, int mode, double omega, const void* r, void* z);
ndiag_status check_device_status(Handle* h);

namespace {

__global__ void bicg_scalars_kernel(double* sc, int first) {
  if (!first && sc[SC_DONE] != 0.0) return;  // stopped: keep the scalars
  if (first) {
    sc[SC_RHO_OLD] = 1.0;
    sc[SC_ALPHA] = 1.0;
    sc[SC_OM] = 1.0;
  } else {
    sc[SC_RHO_OLD] = sc[SC_RHO];
    sc[SC_ALPHA] = sc[SC_RHO] / sc[SC_RV];
    sc[SC_OM] = sc[SC_TT] == 0.0 ? 0.0 : sc[SC_TS] / sc[SC_TT];
  }
  sc[SC_RHO] = sc[SC_RHO_NEXT];
}

// State of a device-resident iteration: running, iterations so far, limit,
// tolerance (absolute ||r||) and its square.
__global__ void loop_init_kernel(double* sc, double it, double maxit, double tol) {
  sc[SC_DONE] = DONE_RUN;
  sc[SC_ITER] = it;
  sc[SC_MAXIT] = maxit;
  sc[SC_TOL] = tol;
  sc[SC_TOL2] = tol * tol;
}

// End of one BiCGSTAB iteration: the tests a host would make after reading the
// scalars, in the same order, so the device decides when to stop. Records the
// iteration (||s||^2, ||r||^2, alpha, omega) when a history buffer is given.
__global__ void bicg_check_kernel(double* sc, double* hist, int cap) {
  if (sc[SC_DONE] != 0.0) return;
  const double rho = sc[SC_RHO], rv = sc[SC_RV], ss = sc[SC_SS], rr = sc[SC_RR];
  const double ts = sc[SC_TS], tt = sc[SC_TT];
  if (rho == 0.0 || rv == 0.0 || !isfinite(ss)) {  // breakdown of the first half step
    sc[SC_DONE] = DONE_BREAK;
    return;
  }
  const double it = sc[SC_ITER] + 1.0;
  sc[SC_ITER] = it;
  if (hist && it <= (double)cap) {
    double* e = hist + 4 * ((int64_t)it - 1);
    e[0] = ss;
    e[1] = rr;
    e[2] = rho / rv;
    e[3] = (ss <= sc[SC_TOL2] || tt == 0.0) ? 0.0 : ts / tt;  // the omega bicg_xr used
  }
  if (ss <= sc[SC_TOL2]) sc[SC_DONE] = DONE_CONV;  // the half step met the tolerance
  else if (!isfinite(rr)) sc[SC_DONE] = DONE_BREAK_NONFINITE;
  else if (sqrt(rr) <= sc[SC_TOL]) sc[SC_DONE] = DONE_CONV;
  else if (tt == 0.0 || ts == 0.0) sc[SC_DONE] = DONE_BREAK_OMEGA;
  else if (it >= sc[SC_MAXIT]) sc[SC_DONE] = DONE_MAXIT;
}

// End of one PCG iteration (after x and r are updated): records
// (||r||^2, alpha) and decides whether to stop.
__global__ void cg_check_kernel(double* sc, double* hist, int cap) {
  if (sc[SC_DONE] != 0.0) return;
  const double pq = sc[SC_PQ], rz = sc[SC_RZ], rr = sc[SC_RR];
  if (pq == 0.0 || rz == 0.0 || !isfinite(rr)) {
    sc[SC_DONE] = DONE_BREAK;
    return;
  }
  const double it = sc[SC_ITER] + 1.0;
  sc[SC_ITER] = it;
  if (hist && it <= (double)cap) {
    double* e = hist + 4 * ((int64_t)it - 1);
    e[0] = rr;
    e[1] = rz / pq;
    e[2] = 0.0;
    e[3] = 0.0;
  }
  if (sqrt(rr) <= sc[SC_TOL]) sc[SC_DONE] = DONE_CONV;
  else if (it >= sc[SC_MAXIT]) sc[SC_DONE] = DONE_MAXIT;
}

template <class T>
__global__ void copy_kernel(int64_t N, const T* s, T* d) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    d[i] = s[i];
}
template <class T>
__global__ void zero_kernel(int64_t N, T* d) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    d[i] = T(0);
}

template <class T>
ndiag_status vcopy(Handle* h, const T* s, T* d) {
  ++h->launches;
  copy_kernel<T><<<h->sm_count * 4, 256, 0, h->stream>>>(h->N, s, d);
  ND_CUDA(cudaGetLastError());
  return NDIAG_OK;
}
template <class T>
ndiag_status vzero(Handle* h, T* d) {
  ++h->launches;
  zero_kernel<T><<<h->sm_count * 4, 256, 0, h->stream>>>(h->N, d);
  ND_CUDA(cudaGetLastError());
  return NDIAG_OK;
}

// Reads the device scalars [SC_BASE, SC_END) into the pinned mirror.
ndiag_status pull(Handle* h) {
  ND_CUDA(cudaMemcpyAsync(h->red_host + SC_BASE, h->red + SC_BASE, sizeof(double) * (SC_END - SC_BASE),
                          cudaMemcpyDeviceToHost, h->stream));
  ND_CUDA(cudaStreamSynchronize(h->stream));
  return NDIAG_OK;
}

struct Prec {
  int kind;
  int mode;
  double omega;
};

ndiag_status apply_prec(Handle* h, const Prec& P, const void* r, void* z, size_t bytes) {
  if (P.kind == NDIAG_PREC_ILU0) return do_ilu_apply(h, r, z);
  if (P.kind == NDIAG_PREC_SSOR) return do_ssor_apply(h, P.mode, P.omega, r, z);
  if (P.kind == NDIAG_PREC_MG) return mg_apply(h, P.omega, (const double*)r, (double*)z);
  ND_CUDA(cudaMemcpyAsync(z, r, bytes, cudaMemcpyDeviceToDevice, h->stream));
  return NDIAG_OK;
}

template <class T>
struct KV {
  T *r, *rh, *p, *v, *ph, *s, *sh, *t;
  T *ps = nullptr, *ss = nullptr;  // pivot-scaled p and s (pre-scaled ILU(0) applies)
};

// Initial residual r = b - A x for the vector type T. fp64: exact residual
// kernel. fp32 inner solves start from x = 0, so r = b.
template <class T>
ndiag_status init_residual(Handle* h, const T* b, const T* x, T* r, double* rr_dev, bool x_is_zero) {
  if (sizeof(T) == 8) return residual64(h, (const double*)b, (const double*)x, (double*)r, rr_dev);
  if (!x_is_zero) {
    set_error("fp32 inner solve must start from zero");
    return NDIAG_EINVAL;
  }
  ND_TRY(vcopy<T>(h, b, r));
  return dots<T>(h, 1, r, r, nullptr, nullptr, nullptr, nullptr, rr_dev, 3);
}

ndiag_status loop_init(Handle* h, int it, int maxit, double tol) {
  ++h->launches;
  loop_init_kernel<<<1, 1, 0, h->stream>>>(h->red, (double)it, (double)maxit, tol);
  ND_CUDA(cudaGetLastError());
  return NDIAG_OK;
}
ndiag_status scalars(Handle* h, int first) {
  ++h->launches;
  bicg_scalars_kernel<<<1, 1, 0, h->stream>>>(h->red, first);
  ND_CUDA(cudaGetLastError());
  return NDIAG_OK;
}

constexpr int CHUNK = 8;  // iterations enqueued between two host reads of the scalars

// Captures CHUNK calls of `body` into one executable graph. The launch counters
// are left as they were and the chunk's counts returned. False if the stream
// cannot be captured here (the caller then launches the chunk directly).
template <class Body>
bool capture_chunk(Handle* h, Body& body, cudaGraphExec_t* exec, int64_t* d_launch, int64_t* d_sweep,
                   double* d_bytes) {
  const int64_t l0 = h->launches, s0 = h->sweep_launches;
  const double b0 = h->sweep_bytes;
  *exec = nullptr;
  if (cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  ndiag_status st = NDIAG_OK;
  for (int k = 0; k < CHUNK && st == NDIAG_OK; ++k) st = body();
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(h->stream, &g);
  *d_launch = h->launches - l0;
  *d_sweep = h->sweep_launches - s0;
  *d_bytes = h->sweep_bytes - b0;
  h->launches = l0;
  h->sweep_launches = s0;
  h->sweep_bytes = b0;
  bool ok = st == NDIAG_OK && e == cudaSuccess && g != nullptr;
  if (ok) ok = cudaGraphInstantiate(exec, g, 0) == cudaSuccess;
  if (g) cudaGraphDestroy(g);
  if (!ok) {
    cudaGetLastError();
    *exec = nullptr;
  }
  return ok;
}

// Runs `body` (the launches of one iteration) in chunks of CHUNK until the
// device stops the iteration, reading the scalars once per chunk. The first
// chunk is launched directly (it also creates every table and buffer that is
// made on first use); with `graph`, the later chunks are one captured CUDA
// graph, replayed. The graph lives for this call. Returns the stop code and
// the iteration count the device reached.
template <class Body>
ndiag_status device_loop(Handle* h, bool graph, int max_iters, Body body, int* done, int* iters) {
  cudaGraphExec_t exec = nullptr;
  int64_t g_launch = 0, g_sweep = 0;
  double g_bytes = 0.0;
  bool first = true, tried = false;
  ndiag_status st = NDIAG_OK;
  // the device stops at the iteration limit at the latest; a chunk more than
  // that means its state word was never set
  const int64_t max_chunks = (int64_t)std::max(max_iters, 0) / CHUNK + 2;
  for (int64_t chunk = 0;; ++chunk) {
    if (chunk > max_chunks) {
      set_error("Krylov iteration: the device did not report a stop within the iteration limit");
      st = NDIAG_EDEVICE;
      break;
    }
    if (!first && graph && !tried) {
      tried = true;
      capture_chunk(h, body, &exec, &g_launch, &g_sweep, &g_bytes);
    }
    if (exec) {
      if (cudaGraphLaunch(exec, h->stream) != cudaSuccess) {
        st = cuda_status(cudaGetLastError(), "cudaGraphLaunch(Krylov chunk)");
        break;
      }
      h->launches += g_launch;
      h->sweep_launches += g_sweep;
      h->sweep_bytes += g_bytes;
    } else {
      for (int k = 0; k < CHUNK && st == NDIAG_OK; ++k) st = body();
      if (st != NDIAG_OK) break;
    }
    first = false;
    st = pull(h);
    if (st != NDIAG_OK) break;
    const double d = h->red_host[SC_DONE];
    if (d != 0.0) {
      *done = (int)d;
      *iters = (int)h->red_host[SC_ITER];
      break;
    }
  }
  if (exec) cudaGraphExecDestroy(exec);
  return st;
}

// Capture is left out while launches are being timed one by one, and for the
// multigrid preconditioner, whose hierarchy is built on the host on first use.
bool graph_allowed(const Handle* h, const Prec& P) { return !h->profiling && P.kind != NDIAG_PREC_MG; }

// BiCGSTAB (van der Vorst 1992), right preconditioned. Stops when the
// recurrence residual meets tol_abs; with `recheck`, then verifies the true
// residual and restarts from it if it is above tol_abs. The iteration runs on
// the device: a check kernel at the end of every iteration makes the stop
// tests (including the half-step exit, taken by bicg_xr with om = 0), and the
// host reads the scalars once per chunk of iterations.
template <class T>
ndiag_status bicgstab(Handle* h, const Prec& P, const T* b, T* x, const KV<T>& V, double tol_abs, int maxit,
                      bool recheck, bool x_is_zero, int* iters) {
  double* sc = h->red;
  const double* hs = h->red_host;
  const size_t vb = sizeof(T) * (size_t)h->N;
  // with the pre-scaled ILU(0) apply the vector kernels also write the
  // pivot-scaled copies p / d~ and s / d~ its forward sweeps read
  const bool pre = V.ps != nullptr;
  const T* inv = pre ? (const T*)ilu_pivot_inverse(h) : nullptr;
  double* hist = sizeof(T) == 8 ? h->hist_dev : nullptr;
  const int cap = hist ? h->hist_cap : 0;
  auto iteration = [&](int first) -> ndiag_status {
    ND_TRY(bicg_p<T>(h, V.r, V.p, V.v, sc, first, inv, V.ps));
    if (pre) ND_TRY(do_ilu_apply_pre(h, V.ps, V.ph));
    else ND_TRY(apply_prec(h, P, V.p, V.ph, vb));
    ND_TRY(spmv_dot<T>(h, V.ph, V.v, V.rh, sc + SC_RV, 1));
    ND_TRY(bicg_s<T>(h, V.r, V.v, V.s, sc, inv, V.ss));
    if (pre) ND_TRY(do_ilu_apply_pre(h, V.ss, V.sh));
    else ND_TRY(apply_prec(h, P, V.s, V.sh, vb));
    ND_TRY(spmv_dot<T>(h, V.sh, V.t, V.s, sc + SC_TS, 2, true));
    ND_TRY(bicg_xr<T>(h, x, V.ph, V.sh, V.r, V.s, V.t, V.rh, sc));
    ++h->launches;
    bicg_check_kernel<<<1, 1, 0, h->stream>>>(sc, hist, cap);
    ND_CUDA(cudaGetLastError());
    return scalars(h, 0);  // the next iteration's alpha, omega, rho
  };
  int it = 0;
  for (;;) {
    ND_TRY(init_residual<T>(h, b, x, V.r, sc + SC_R0, x_is_zero));
    ND_TRY(pull(h));
    if (std::sqrt(hs[SC_R0]) <= tol_abs) break;
    if (it >= maxit) {
      *iters = it;
      return NDIAG_ENOCONV;
    }
    ND_TRY(vcopy<T>(h, V.r, V.rh));
    ND_TRY(dots<T>(h, 1, V.rh, V.r, nullptr, nullptr, nullptr, nullptr, sc + SC_RHO_NEXT, 1));
    ND_TRY(loop_init(h, it, maxit, tol_abs));
    ND_TRY(scalars(h, 1));
    ND_TRY(iteration(1));
    int done = DONE_RUN;
    ND_TRY(device_loop(h, graph_allowed(h, P), maxit - it, [&] { return iteration(0); }, &done, &it));
    *iters = it;
    if (done == DONE_MAXIT) return NDIAG_ENOCONV;
    if (done == DONE_BREAK) {
      set_error("BiCGSTAB breakdown");
      return NDIAG_EBREAKDOWN;
    }
    if (done == DONE_BREAK_NONFINITE) {
      set_error("BiCGSTAB breakdown (non-finite residual)");
      return NDIAG_EBREAKDOWN;
    }
    if (done == DONE_BREAK_OMEGA) {
      set_error("BiCGSTAB breakdown (omega = 0)");
      return NDIAG_EBREAKDOWN;
    }
    if (!recheck) break;  // DONE_CONV
    x_is_zero = false;
  }
  *iters = it;
  return NDIAG_OK;
}

// Preconditioned CG (Saad Alg. 9.1), same stop rule, the same device-resident
// loop.
template <class T>
ndiag_status pcg(Handle* h, const Prec& P, const T* b, T* x, const KV<T>& V, double tol_abs, int maxit,
                 bool recheck, bool x_is_zero, int* iters) {
  double* sc = h->red;
  const double* hs = h->red_host;
  const size_t vb = sizeof(T) * (size_t)h->N;
  T *r = V.r, *z = V.s, *p = V.p, *q = V.v;
  double* hist = sizeof(T) == 8 ? h->hist_dev : nullptr;
  const int cap = hist ? h->hist_cap : 0;
  auto iteration = [&]() -> ndiag_status {
    ND_TRY(spmv_dot<T>(h, p, q, p, sc + SC_PQ, 2));
    ND_TRY(cg_xr<T>(h, x, p, r, q, sc));
    ++h->launches;
    cg_check_kernel<<<1, 1, 0, h->stream>>>(sc, hist, cap);
    ND_CUDA(cudaGetLastError());
    ND_TRY(apply_prec(h, P, r, z, vb));
    ND_TRY(dots<T>(h, 1, r, z, nullptr, nullptr, nullptr, nullptr, sc + SC_RZ_NEW, 1));
    ND_TRY(cg_p<T>(h, z, p, sc, 0));
    return copy_scalar(h, sc, SC_RZ, SC_RZ_NEW);
  };
  int it = 0;
  for (;;) {
    ND_TRY(init_residual<T>(h, b, x, r, sc + SC_R0, x_is_zero));
    ND_TRY(pull(h));
    if (std::sqrt(hs[SC_R0]) <= tol_abs) break;
    if (it >= maxit) {
      *iters = it;
      return NDIAG_ENOCONV;
    }
    ND_TRY(loop_init(h, it, maxit, tol_abs));  // before cg_p, which skips once stopped
    ND_TRY(apply_prec(h, P, r, z, vb));
    ND_TRY(dots<T>(h, 1, r, z, nullptr, nullptr, nullptr, nullptr, sc + SC_RZ, 1));
    ND_TRY(cg_p<T>(h, z, p, sc, 1));
    int done = DONE_RUN;
    ND_TRY(device_loop(h, graph_allowed(h, P), maxit - it, iteration, &done, &it));
    *iters = it;
    if (done == DONE_MAXIT) return NDIAG_ENOCONV;
    if (done != DONE_CONV) {
      set_error("PCG breakdown");
      return NDIAG_EBREAKDOWN;
    }
    if (!recheck) break;
    x_is_zero = false;
  }
  *iters = it;
  return NDIAG_OK;
}

// Stationary SOR iteration with the schedule t = 0, 1, 2, ...: stops at the
// first iterate whose true residual meets tol_abs (checked after every sweep).
template <class T>
ndiag_status stationary(Handle* h, int mode, const double* omega, const T* b, T* x, T* xalt, T* r,
                        double tol_abs, int maxit, bool x_is_zero, int* iters) {
  double* sc = h->red;
  const double* hs = h->red_host;
  ND_TRY(init_residual<T>(h, b, x, r, sc + SC_R0, x_is_zero));
  ND_TRY(pull(h));
  double rel = std::sqrt(hs[SC_R0]);
  int it = 0;
  T* cur = x;
  T* nxt = xalt;
  while (rel > tol_abs && it < maxit) {
    if (h->dim == 3)
      ND_TRY(launch_sweep3d(h, KIND_SOR, mode, it, omega, h->sor, b, cur, nxt, 1.0, false));
    else if (h->stencil == 9)
      ND_TRY(launch_sweep9(h, KIND_SOR, mode, it, omega, h->sor, b, cur, nxt, 1.0));
    else
      ND_TRY(launch_sweep2d(h, KIND_SOR, mode, it, omega, h->sor, b, cur, nxt));
    ++it;
    if (sizeof(T) == 8) {
      ND_TRY(residual64(h, (const double*)b, (const double*)nxt, (double*)r, sc + SC_R0));
    } else {
      ND_TRY(spmv_any<T>(h, nxt, r));
      // r = b - A x in fp32 with the norm in fp64 (inner solve only)
      ND_TRY(dots<T>(h, 1, r, r, nullptr, nullptr, nullptr, nullptr, sc + SC_R0, 3));
      set_error("fp32 stationary inner residual not supported");
      return NDIAG_EINVAL;
    }
    ND_TRY(pull(h));
    rel = std::sqrt(hs[SC_R0]);
    T* tmp = cur;
    cur = nxt;
    nxt = tmp;
  }
  if (cur != x) ND_TRY(vcopy<T>(h, cur, x));
  *iters = it;
  return rel <= tol_abs ? NDIAG_OK : NDIAG_ENOCONV;
}

ndiag_status ensure_kws(Handle* h, size_t bytes) {
  if (h->kws.bytes >= bytes) return NDIAG_OK;
  dev_free(h->kws.p, h->kws.bytes, h->stream);
  h->kws.p = dev_alloc(bytes, h->stream);
  h->kws.bytes = h->kws.p ? bytes : 0;
  return h->kws.p ? NDIAG_OK : NDIAG_ENOMEM;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <class T>
KV<T> carve(char*& cur, int64_t N) {
  KV<T> V;
  T** slots[8] = {&V.r, &V.rh, &V.p, &V.v, &V.ph, &V.s, &V.sh, &V.t};
  for (T** s : slots) {
    *s = (T*)cur;
    cur += ((sizeof(T) * (size_t)N + 255) / 256) * 256;
  }
  return V;
}

}  // namespace
}  // namespace nd

using namespace nd;

extern "C" ndiag_status krylov_solve(ndiag* h, int method, int precond, int mode, const double* omega,
                                     double rtol, int maxit, const double* b, double* x,
                                     ndiag_solve_info* info) {
  const auto t0 = std::chrono::steady_clock::now();
  if (!h || !b || !x || !omega || !(rtol > 0.0) || maxit < 0) return NDIAG_EINVAL;
  if (method < NDIAG_PCG || method > NDIAG_STATIONARY) return NDIAG_EINVAL;
  if (precond < NDIAG_PREC_NONE || precond > NDIAG_PREC_MG) return NDIAG_EINVAL;
  if (method != NDIAG_STATIONARY && precond == NDIAG_PREC_MG &&
      (!((h->dim == 2 && h->stencil == 5) || (h->dim == 3 && h->stencil == 7)) || h->precision != NDIAG_FP64 ||
       mode != NDIAG_DECOMPOSED || !(omega[0] > 0.0 && omega[0] < 2.0))) {
    set_error("the multigrid preconditioner needs a 2D 5-point or 3D 7-point fp64 handle, DECOMPOSED mode "
              "and 0 < omega < 2");
    return NDIAG_EINVAL;
  }
  if (mode != NDIAG_NATURAL && mode != NDIAG_DECOMPOSED) return NDIAG_EINVAL;
  if (method != NDIAG_STATIONARY && precond == NDIAG_PREC_ILU0 && h->ilu_mode < 0) {
    set_error("ILU(0) preconditioner requested before ilu0_factor");
    return NDIAG_ESTATE;
  }
  const int64_t N = h->N;
  const size_t v64 = ((sizeof(double) * (size_t)N + 255) / 256) * 256;
  const size_t v32 = ((sizeof(float) * (size_t)N + 255) / 256) * 256;
  const bool fp64 = h->precision == NDIAG_FP64;
  const bool dev_b = is_device_ptr(b), dev_x = is_device_ptr(x);
  // fp64 vectors: 8 Krylov + alt + b copy + x copy ; fp32: 8 inner + e + r64 + b + x
  const size_t need = fp64 ? v64 * 13 : v32 * 9 + v64 * 3;  // fp64: + the two pre-scaled vectors
  ND_TRY(ensure_kws(h, need));
  char* cur = (char*)h->kws.p;
  Prec P{precond, mode, omega[0]};
  int iters = 0, outer = 0;
  ndiag_status st = NDIAG_OK;
  double bnorm = 0.0, relres = 0.0;
  if (fp64) {
    KV<double> V = carve<double>(cur, N);
    if (method == NDIAG_BICGSTAB && precond == NDIAG_PREC_ILU0 && ilu_prescaled_ok(h)) {
      V.ps = (double*)cur;
      V.ss = (double*)(cur + v64);
    }
    cur += 2 * v64;
    double* xalt = (double*)cur;
    cur += v64;
    double* bd = dev_b ? (double*)b : (double*)cur;
    cur += v64;
    double* xd = dev_x ? x : (double*)cur;
    if (!dev_b) ND_CUDA(cudaMemcpyAsync(bd, b, sizeof(double) * N, cudaMemcpyHostToDevice, h->stream));
    if (!dev_x) ND_CUDA(cudaMemcpyAsync(xd, x, sizeof(double) * N, cudaMemcpyHostToDevice, h->stream));
    ND_TRY(dots<double>(h, 1, bd, bd, nullptr, nullptr, nullptr, nullptr, h->red + SC_BB, 3));
    ND_TRY(pull(h));
    bnorm = std::sqrt(h->red_host[SC_BB]);
    const double tol = rtol * (bnorm > 0 ? bnorm : 1.0);
    if (method == NDIAG_BICGSTAB) st = bicgstab<double>(h, P, bd, xd, V, tol, maxit, true, false, &iters);
    else if (method == NDIAG_PCG) st = pcg<double>(h, P, bd, xd, V, tol, maxit, true, false, &iters);
    else st = stationary<double>(h, mode, omega, bd, xd, xalt, V.r, tol, maxit, false, &iters);
    outer = 1;
    if (st == NDIAG_OK || st == NDIAG_ENOCONV) {
      ndiag_status s2 = residual64(h, bd, xd, V.r, h->red + SC_R0);
      if (s2 == NDIAG_OK) s2 = pull(h);
      if (s2 != NDIAG_OK) st = s2;
      relres = std::sqrt(h->red_host[SC_R0]) / (bnorm > 0 ? bnorm : 1.0);
    }
    if (!dev_x) ND_CUDA(cudaMemcpyAsync(x, xd, sizeof(double) * N, cudaMemcpyDeviceToHost, h->stream));
  } else {
    KV<float> V = carve<float>(cur, N);
    float* e = (float*)cur;
    cur += v32;
    double* r64 = (double*)cur;
    cur += v64;
    double* bd = dev_b ? (double*)b : (double*)cur;
    cur += v64;
    double* xd = dev_x ? x : (double*)cur;
    if (!dev_b) ND_CUDA(cudaMemcpyAsync(bd, b, sizeof(double) * N, cudaMemcpyHostToDevice, h->stream));
    if (!dev_x) ND_CUDA(cudaMemcpyAsync(xd, x, sizeof(double) * N, cudaMemcpyHostToDevice, h->stream));
    ND_TRY(dots<double>(h, 1, bd, bd, nullptr, nullptr, nullptr, nullptr, h->red + SC_BB, 3));
    ND_TRY(pull(h));
    bnorm = std::sqrt(h->red_host[SC_BB]);
    const double tol = rtol * (bnorm > 0 ? bnorm : 1.0);
    // inner tolerance: aim at the outer tolerance with one inner solve, but
    // not below 1e-6 relative (where fp32 sweeps and vectors stop gaining), and
    // never looser than 1e-3
    const double inner_floor = 1e-6, inner_ceil = 1e-3;
    int max_outer = 60;
    for (;;) {
      // fp64 residual of the outer iterate, delivered in fp32 to the inner solve
      ND_TRY(residual64_to32(h, bd, xd, V.t, h->red + SC_R0));
      ND_TRY(pull(h));
      const double rn = std::sqrt(h->red_host[SC_R0]);
      relres = rn / (bnorm > 0 ? bnorm : 1.0);
      if (rn <= tol) break;
      if (outer >= max_outer || iters >= maxit) {
        st = NDIAG_ENOCONV;
        break;
      }
      ++outer;
      ND_TRY(vzero<float>(h, e));
      int it_in = 0;
      // the inner solve's right-hand side lives in V.t; copy it out first
      ND_TRY(vcopy<float>(h, V.t, (float*)r64));
      const double tol_in = std::min(inner_ceil, std::max(inner_floor, 0.5 * tol / rn)) * rn;
      ndiag_status si;
      if (method == NDIAG_PCG) si = pcg<float>(h, P, (float*)r64, e, V, tol_in, maxit - iters, false, true, &it_in);
      else if (method == NDIAG_BICGSTAB)
        si = bicgstab<float>(h, P, (float*)r64, e, V, tol_in, maxit - iters, false, true, &it_in);
      else {
        set_error("stationary method with fp32 precision is not supported");
        return NDIAG_EINVAL;
      }
      iters += it_in;
      if (si != NDIAG_OK && si != NDIAG_ENOCONV) {
        st = si;
        break;
      }
      ND_TRY(add_to(h, xd, e));
    }
    if (!dev_x) ND_CUDA(cudaMemcpyAsync(x, xd, sizeof(double) * N, cudaMemcpyDeviceToHost, h->stream));
  }
  // the per-iteration record: squared norms become norms relative to ||b||
  const int nrec = std::min(iters, h->hist_cap);
  if (fp64 && h->hist_user && nrec > 0 && method != NDIAG_STATIONARY)
    ND_CUDA(cudaMemcpyAsync(h->hist_user, h->hist_dev, sizeof(double) * 4 * (size_t)nrec, cudaMemcpyDeviceToHost,
                            h->stream));
  ND_CUDA(cudaStreamSynchronize(h->stream));
  if (fp64 && h->hist_user && nrec > 0 && method != NDIAG_STATIONARY) {
    const double bn = bnorm > 0 ? bnorm : 1.0;
    for (int k = 0; k < nrec; ++k) {
      double* e = h->hist_user + 4 * (size_t)k;
      e[0] = std::sqrt(e[0]) / bn;
      if (method == NDIAG_BICGSTAB) e[1] = std::sqrt(e[1]) / bn;
    }
  }
  ndiag_status ds = check_device_status(h);
  if (ds == NDIAG_OK && P.kind == NDIAG_PREC_MG && method != NDIAG_STATIONARY) ds = mg_check(h);
  if (ds != NDIAG_OK) st = ds;
  if (info) {
    info->iterations = iters;
    info->outer = outer;
    info->relres = relres;
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    info->status = st;
  }
  return st;
}

extern "C" ndiag_status ndiag_set_history(ndiag* h, double* out, int capacity) {
  if (!h || capacity < 0) return NDIAG_EINVAL;
  dev_free(h->hist_dev, sizeof(double) * 4 * (size_t)h->hist_cap, h->stream);
  h->hist_dev = nullptr;
  h->hist_cap = 0;
  h->hist_user = nullptr;
  if (!out || capacity == 0) return NDIAG_OK;
  h->hist_dev = (double*)dev_alloc(sizeof(double) * 4 * (size_t)capacity, h->stream);
  if (!h->hist_dev) return NDIAG_ENOMEM;
  h->hist_cap = capacity;
  h->hist_user = out;
  return NDIAG_OK;
}
