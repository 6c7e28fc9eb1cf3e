// C ABI entry points: handle life cycle, storage, sweeps and ILU(0).
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>

#include "blas.h"
#include "internal.h"

namespace nd {

static thread_local std::string g_last_error;
static ndiag_alloc_fn g_alloc = nullptr;
static ndiag_free_fn g_free = nullptr;
static void* g_alloc_ctx = nullptr;
static std::mutex g_alloc_mu;
static thread_local bool g_tls_plain_alloc = false;  // this thread ignores the allocator hooks

void use_plain_allocator_on_this_thread(bool on) { g_tls_plain_alloc = on; }

void set_error(const std::string& msg) { g_last_error = msg; }

ndiag_status cuda_status(cudaError_t e, const char* what) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  if (e == cudaErrorMemoryAllocation) return NDIAG_ENOMEM;
  return NDIAG_EDEVICE;
}

void* dev_alloc(size_t bytes, cudaStream_t s) {
  if (bytes == 0) bytes = 16;
  ndiag_alloc_fn a;
  void* ctx;
  {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    a = g_tls_plain_alloc ? nullptr : g_alloc;
    ctx = g_alloc_ctx;
  }
  if (a) return a(bytes, (void*)s, ctx);
  void* p = nullptr;
  if (cudaMallocAsync(&p, bytes, s) != cudaSuccess) {
    cudaGetLastError();
    set_error("device allocation failed");
    return nullptr;
  }
  return p;
}

void dev_free(void* p, size_t bytes, cudaStream_t s) {
  if (!p) return;
  ndiag_free_fn f;
  void* ctx;
  {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    f = g_tls_plain_alloc ? nullptr : g_free;
    ctx = g_alloc_ctx;
  }
  if (f) {
    f(p, bytes, (void*)s, ctx);
    return;
  }
  cudaFreeAsync(p, s);
}

int base_corner(int dim, int64_t t) {
  if (dim == 1) return (int)(t & 1);
  const int period = 1 << dim;
  const int tt = (int)(((t % period) + period) % period);
  const int all = period - 1;
  int c = all ^ (tt >> 1);
  if (tt & 1) c = all ^ c;
  return c;
}

ndiag_status launch_ilu_factor2d_into(Handle* h, int mode, double* out);

int prof_begin(Handle* h) {
  if (!h->profiling) return -1;
  ProfRec r;
  for (cudaEvent_t* e : {&r.a, &r.b}) {
    if (!h->ev_pool.empty()) {
      *e = h->ev_pool.back();
      h->ev_pool.pop_back();
    } else if (cudaEventCreate(e) != cudaSuccess) {
      cudaGetLastError();
      return -1;
    }
  }
  cudaEventRecord(r.a, h->stream);
  h->prof.push_back(r);
  return (int)h->prof.size() - 1;
}

void prof_end(Handle* h, int slot, double bytes) {
  h->sweep_bytes += bytes;
  if (slot < 0) return;
  h->prof[slot].bytes = bytes;
  cudaEventRecord(h->prof[slot].b, h->stream);
}

static void prof_collect(Handle* h) {
  for (ProfRec& r : h->prof) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) h->sweep_ms += ms;
    else cudaGetLastError();
    h->ev_pool.push_back(r.a);
    h->ev_pool.push_back(r.b);
  }
  h->prof.clear();
}

namespace {

template <class TC>
__global__ void scaled_set_kernel(int64_t N, int s, const double* A, const double* piv, TC* out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const double p = piv ? piv[i] : A[i];
    out[i] = (TC)(1.0 / p);
    for (int e = 1; e < s; ++e) out[(size_t)e * N + i] = (TC)(A[(size_t)e * N + i] / p);
  }
}
template <class TC>
__global__ void convert_matrix_kernel(int64_t n, const double* A, TC* out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (TC)A[i];
}

size_t coef_size(int precision) {
  return precision == NDIAG_FP64 ? 8 : precision == NDIAG_FP32 ? 4 : 2;
}

}  // namespace

ndiag_status build_scaled(Handle* h, ScaledSet& set, const double* piv) { return build_scaled_from(h, set, h->A64, piv); }

ndiag_status build_scaled_from(Handle* h, ScaledSet& set, const double* A, const double* piv) {
  const size_t bytes = coef_size(h->precision) * (size_t)h->stencil * (size_t)h->N;
  if (!set.base) {
    set.base = dev_alloc(bytes, h->stream);
    if (!set.base) return NDIAG_ENOMEM;
    set.bytes = bytes;
  }
  const int grid = h->sm_count * 4;
  ++h->launches;
  ++set.version;
  switch (h->precision) {
    case NDIAG_FP64:
      scaled_set_kernel<double><<<grid, 256, 0, h->stream>>>(h->N, h->stencil, A, piv, (double*)set.base);
      break;
    case NDIAG_FP32:
      scaled_set_kernel<float><<<grid, 256, 0, h->stream>>>(h->N, h->stencil, A, piv, (float*)set.base);
      break;
    default:
      scaled_set_kernel<__half><<<grid, 256, 0, h->stream>>>(h->N, h->stencil, A, piv, (__half*)set.base);
  }
  ND_CUDA(cudaGetLastError());
  return NDIAG_OK;
}

namespace {

ndiag_status check_status(Handle* h) {
  DevStatus st{};
  ND_CUDA(cudaMemcpyAsync(&st, h->status, sizeof(st), cudaMemcpyDeviceToHost, h->stream));
  ND_CUDA(cudaStreamSynchronize(h->stream));
  if (st.timeout) {
    set_error("a bounded device-side wait timed out");
    cudaMemsetAsync(h->status, 0, sizeof(DevStatus), h->stream);
    return NDIAG_ETIMEOUT;
  }
  if (st.zero_pivot) {
    set_error("zero pivot in ILU(0)");
    cudaMemsetAsync(h->status, 0, sizeof(DevStatus), h->stream);
    return NDIAG_EBREAKDOWN;
  }
  return NDIAG_OK;
}

}  // namespace

ndiag_status ensure_tmp(Handle* h) {
  if (h->tmp) return NDIAG_OK;
  h->tmp = dev_alloc(h->vec_bytes, h->stream);
  if (!h->tmp) return NDIAG_ENOMEM;
  h->tmp_bytes = h->vec_bytes;
  return NDIAG_OK;
}

ndiag_status do_ilu_apply(Handle* h, const void* r, void* z) {
  if (h->ilu_mode < 0) {
    set_error("ilu0_apply before ilu0_factor");
    return NDIAG_ESTATE;
  }
  ND_TRY(ensure_tmp(h));
  const int64_t tf = fwd_phase(h->dim);
  // (D~ + L_J) y = r ; (D~ + U_J) z = D~ y   (U_J = implicit set of the reverse phase)
  const int back = h->ilu_mode == NDIAG_NATURAL ? (int)MODE_NATURAL_REV : h->ilu_mode;
  if (h->dim == 3) {
    ND_TRY(launch_sweep3d(h, KIND_TRI_SCALED, h->ilu_mode, tf, nullptr, h->ilu, r, nullptr, h->tmp, 1.0, false));
    return launch_sweep3d(h, KIND_TRI_UNIT, back, tf ^ 1, nullptr, h->ilu, h->tmp, nullptr, z, 1.0, false);
  }
  if (h->stencil == 9) {
    ND_TRY(launch_sweep9(h, KIND_TRI_SCALED, h->ilu_mode, tf, nullptr, h->ilu, r, nullptr, h->tmp, 1.0));
    return launch_sweep9(h, KIND_TRI_UNIT, back, tf ^ 1, nullptr, h->ilu, h->tmp, nullptr, z, 1.0);
  }
  ND_TRY(launch_sweep2d(h, KIND_TRI_SCALED, h->ilu_mode, tf, nullptr, h->ilu, r, nullptr, h->tmp));
  ND_TRY(launch_sweep2d(h, KIND_TRI_UNIT, back, tf ^ 1, nullptr, h->ilu, h->tmp, nullptr, z));
  return NDIAG_OK;
}

// The ILU(0) apply of a right-hand side given already scaled by the pivots,
// rs = d~^-1 .* r (2D 5-point): the forward sweep then solves the unit form
// (I + D~^-1 L_J) y = rs, operation for operation the same values as
// do_ilu_apply, with the scaling done by the caller's vector kernel.
bool ilu_prescaled_ok(const Handle* h) {
  return h->dim == 2 && h->stencil == 5 && h->precision == NDIAG_FP64 && h->ilu_mode == NDIAG_DECOMPOSED;
}
const double* ilu_pivot_inverse(const Handle* h) { return (const double*)h->ilu.base; }
ndiag_status do_ilu_apply_pre(Handle* h, const void* rs, void* z) {
  if (!ilu_prescaled_ok(h)) {
    set_error("pre-scaled ILU(0) apply needs a decomposed 2D 5-point fp64 factorisation");
    return NDIAG_ESTATE;
  }
  ND_TRY(ensure_tmp(h));
  const int64_t tf = fwd_phase(h->dim);
  ND_TRY(launch_sweep2d(h, KIND_TRI_UNIT, h->ilu_mode, tf, nullptr, h->ilu, rs, nullptr, h->tmp));
  return launch_sweep2d(h, KIND_TRI_UNIT, h->ilu_mode, tf ^ 1, nullptr, h->ilu, h->tmp, nullptr, z);
}

ndiag_status check_device_status(Handle* h) { return check_status(h); }

// z = w(2-w) (D + w L_J^T)^-1 D (D + w L_J)^-1 r   (forward phase J)
ndiag_status do_ssor_apply(Handle* h, int mode, double omega, const void* r, void* z) {
  if (!(omega > 0.0 && omega < 2.0)) {
    set_error("SSOR needs 0 < omega < 2");
    return NDIAG_EINVAL;
  }
  if (h->stencil == 9) {
    set_error("SSOR is not available for the 9-point stencil (use SOR or ILU(0))");
    return NDIAG_EINVAL;
  }
  ND_TRY(ensure_tmp(h));
  if (!h->sorT.base) ND_TRY(build_scaled_transposed(h, h->sorT));
  const double om[8] = {omega, omega, omega, omega, omega, omega, omega, omega};
  const int64_t tf = fwd_phase(h->dim);
  if (h->dim == 3) {
    // forward: tmp = w(2-w) (D + w L_J)^-1 r ; then (D + w L_J^T) z = D tmp
    ND_TRY(launch_sweep3d(h, KIND_TRI_SCALED, mode, tf, om, h->sor, r, nullptr, h->tmp, omega * (2.0 - omega),
                          false));
    return launch_sweep3d(h, KIND_TRI_UNIT, mode, tf, om, h->sorT, h->tmp, nullptr, z, 1.0, true);
  }
  // forward: tmp = w(2-w) (D + w L_J)^-1 r
  ND_TRY(launch_sweep2d_ex(h, KIND_TRI_SCALED, mode, tf, om, h->sor, r, nullptr, h->tmp,
                           omega * (2.0 - omega), false));
  // backward: (D + w L_J^T) z = D tmp, interiors in the reversed frame, then
  // the coupled interface pairs and corners
  const int back = mode == NDIAG_NATURAL ? (int)MODE_NATURAL_REV : mode;
  ND_TRY(launch_sweep2d_ex(h, KIND_TRI_UNIT, back, tf ^ 1, om, h->sorT, h->tmp, nullptr, z, 1.0, true));
  return launch_ssor_edges2d(h, mode, omega, h->tmp, z);
}

}  // namespace nd

using namespace nd;

extern "C" {

ndiag_status ndiag_set_allocator(ndiag_alloc_fn alloc, ndiag_free_fn release, void* ctx) {
  if ((alloc == nullptr) != (release == nullptr)) return NDIAG_EINVAL;
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  g_alloc = alloc;
  g_free = release;
  g_alloc_ctx = ctx;
  return NDIAG_OK;
}

const char* ndiag_last_error(void) { return g_last_error.c_str(); }

ndiag_status ndiag_create(ndiag** out, int dim, const int64_t n[3], int stencil, const double* diags,
                          const int sub[3], int precision, void* cuda_stream) {
  if (!out) return NDIAG_EINVAL;
  *out = nullptr;
  if (!n || !diags || !sub) return NDIAG_EINVAL;
  if (!((dim == 2 && (stencil == 5 || stencil == 9)) || (dim == 3 && stencil == 7))) {
    set_error("unsupported dim/stencil");
    return NDIAG_EINVAL;
  }
  if (precision < NDIAG_FP64 || precision > NDIAG_FP32_D16) return NDIAG_EINVAL;
  int64_t N = 1;
  for (int a = 0; a < dim; ++a) {
    if (n[a] < 1 || n[a] > (1 << 20) || sub[a] < 1 || sub[a] > n[a]) {
      set_error("bad grid size or subdomain count");
      return NDIAG_EINVAL;
    }
    N *= n[a];
  }
  if (N > ((int64_t)1 << 31) - 1) {
    set_error("grid too large (N must fit in int32)");
    return NDIAG_EINVAL;
  }
  for (int64_t i = 0; i < N; ++i)
    if (!(diags[i] > 0.0)) {
      set_error("diagonal entries must be positive");
      return NDIAG_EINVAL;
    }

  ndiag* h = new (std::nothrow) ndiag();
  if (!h) return NDIAG_ENOMEM;
  h->dim = dim;
  h->stencil = stencil;
  h->precision = precision;
  for (int a = 0; a < 3; ++a) {
    h->n[a] = a < dim ? n[a] : 1;
    h->sub[a] = a < dim ? sub[a] : 1;
  }
  h->N = N;
  h->stream = (cudaStream_t)cuda_stream;
  h->vec_bytes = (size_t)N * (precision == NDIAG_FP64 ? 8 : 4);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) {
    delete h;
    return cuda_status(e, "cudaGetDevice");
  }
  const size_t abytes = sizeof(double) * (size_t)stencil * (size_t)N;
  h->A64 = (double*)dev_alloc(abytes, h->stream);
  h->status = (DevStatus*)dev_alloc(sizeof(DevStatus), h->stream);
  h->red_bytes = reduce_bytes(h);
  h->red = (double*)dev_alloc(h->red_bytes, h->stream);
  if (!h->A64 || !h->status || !h->red) {
    ndiag_destroy(h);
    return NDIAG_ENOMEM;
  }
  if (cudaMallocHost(&h->red_host, sizeof(double) * RED_RES) != cudaSuccess) {
    cudaGetLastError();
    h->red_host = nullptr;
    ndiag_destroy(h);
    return NDIAG_ENOMEM;
  }
  ndiag_status st = NDIAG_OK;
  e = cudaMemcpyAsync(h->A64, diags, abytes, cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->status, 0, sizeof(DevStatus), h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->red, 0, h->red_bytes, h->stream);
  if (e != cudaSuccess) st = cuda_status(e, "upload");
  if (st == NDIAG_OK && precision != NDIAG_FP64) {
    h->Alo = dev_alloc(sizeof(float) * (size_t)stencil * (size_t)N, h->stream);
    if (!h->Alo) st = NDIAG_ENOMEM;
    else {
      ++h->launches;
      convert_matrix_kernel<float><<<h->sm_count * 4, 256, 0, h->stream>>>((int64_t)stencil * N, h->A64,
                                                                          (float*)h->Alo);
      e = cudaGetLastError();
      if (e != cudaSuccess) st = cuda_status(e, "convert");
    }
  }
  if (st == NDIAG_OK) st = build_scaled(h, h->sor, nullptr);
  if (st == NDIAG_OK) {
    e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) st = cuda_status(e, "create");
  }
  if (st != NDIAG_OK) {
    ndiag_destroy(h);
    return st;
  }
  *out = h;
  return NDIAG_OK;
}

void ndiag_destroy(ndiag* h) {
  if (!h) return;
  cudaStream_t s = h->stream;
  mg_free(h);
  w9pack_free(h);
  dev_free(h->A64, 0, s);
  dev_free(h->Alo, 0, s);
  dev_free(h->sor.base, h->sor.bytes, s);
  dev_free(h->ilu.base, h->ilu.bytes, s);
  dev_free(h->sorT.base, h->sorT.bytes, s);
  dev_free(h->sor.lev, h->sor.lev_bytes, s);
  dev_free(h->ilu.lev, h->ilu.lev_bytes, s);
  dev_free(h->sorT.lev, h->sorT.lev_bytes, s);
  dev_free(h->vcount, h->vcount_bytes, s);
  dev_free(h->sync, h->sync_bytes, s);
  dev_free(h->twin_hand, h->twin_hand_bytes, s);
  for (LineTable& t : h->line_tables) dev_free(t.buf, t.bytes, s);
  dev_free(h->status, sizeof(DevStatus), s);
  dev_free(h->kws.p, h->kws.bytes, s);
  dev_free(h->red, h->red_bytes, s);
  dev_free(h->tmp, h->tmp_bytes, s);
  dev_free(h->hist_dev, sizeof(double) * 4 * (size_t)h->hist_cap, s);
  cudaStreamSynchronize(s);
  for (ProfRec& r : h->prof) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
  if (h->red_host) cudaFreeHost(h->red_host);
  delete h;
}

int64_t ndiag_cells(const ndiag* h) { return h ? h->N : 0; }

ndiag_status ndiag_profile(ndiag* h, int enable) {
  if (!h) return NDIAG_EINVAL;
  ND_CUDA(cudaStreamSynchronize(h->stream));
  prof_collect(h);
  h->launches = 0;
  h->sweep_launches = 0;
  h->sweep_ms = 0.0;
  h->sweep_bytes = 0.0;
  h->profiling = enable != 0;
  return NDIAG_OK;
}

ndiag_status ndiag_set_wavefront(ndiag* h, int on) {
  if (!h) return NDIAG_EINVAL;
  h->w9_wave = on != 0;
  h->w3_wave = on != 0;
  return NDIAG_OK;
}

ndiag_status ndiag_read_counters(ndiag* h, ndiag_counters* out) {
  if (!h || !out) return NDIAG_EINVAL;
  ND_CUDA(cudaStreamSynchronize(h->stream));
  prof_collect(h);
  out->launches = h->launches;
  out->sweep_launches = h->sweep_launches;
  out->sweep_ms = h->sweep_ms;
  out->sweep_bytes = h->sweep_bytes;
  return NDIAG_OK;
}
int ndiag_precision(const ndiag* h) { return h ? h->precision : -1; }

ndiag_status sor_sweep(ndiag* h, int mode, const double* omega, int64_t t, const void* b, const void* x_old,
                       void* x_new) {
  if (!h || !omega || !b || !x_old || !x_new || x_old == x_new) return NDIAG_EINVAL;
  if (mode != NDIAG_NATURAL && mode != NDIAG_DECOMPOSED) return NDIAG_EINVAL;
  if (h->dim == 3) return launch_sweep3d(h, KIND_SOR, mode, t, omega, h->sor, b, x_old, x_new, 1.0, false);
  if (h->stencil == 9) return launch_sweep9(h, KIND_SOR, mode, t, omega, h->sor, b, x_old, x_new, 1.0);
  return launch_sweep2d(h, KIND_SOR, mode, t, omega, h->sor, b, x_old, x_new);
}

ndiag_status ilu0_factor(ndiag* h, int mode) {
  if (!h || (mode != NDIAG_NATURAL && mode != NDIAG_DECOMPOSED && mode != NDIAG_DECOMPOSED_FULL))
    return NDIAG_EINVAL;
  // on 5/7-point matrices the full factor of every subdomain block changes
  // only the pivots, exactly as the decomposed one does
  if (mode == NDIAG_DECOMPOSED_FULL && h->stencil != 9) mode = NDIAG_DECOMPOSED;
  if (h->stencil == 9 && mode != NDIAG_DECOMPOSED) {
    // true ILU(0) with modified off-diagonals, as a 9 x N matrix (D + L') D^-1 (D + U'):
    // of the whole lexicographic order, or of every subdomain block in its sweep order
    const size_t fb = sizeof(double) * 9 * (size_t)h->N;
    double* F = (double*)dev_alloc(fb, h->stream);
    if (!F) return NDIAG_ENOMEM;
    ndiag_status st = mode == NDIAG_NATURAL ? launch_ilu_factor9_natural(h, F) : launch_ilu_factor9_full(h, F);
    if (st == NDIAG_OK) st = build_scaled_from(h, h->ilu, F, F);
    dev_free(F, fb, h->stream);
    if (st == NDIAG_OK) st = check_status(h);
    // the full factor is applied by the decomposed sweeps
    h->ilu_mode = st == NDIAG_OK ? (mode == NDIAG_NATURAL ? NDIAG_NATURAL : NDIAG_DECOMPOSED) : -1;
    return st;
  }
  double* dt = (double*)dev_alloc(sizeof(double) * (size_t)h->N, h->stream);
  if (!dt) return NDIAG_ENOMEM;
  ndiag_status st = h->dim == 3        ? launch_ilu_factor3d_into(h, mode, dt)
                    : h->stencil == 9 ? launch_ilu_factor9_into(h, mode, dt)
                                      : launch_ilu_factor2d_into(h, mode, dt);
  if (st == NDIAG_OK) st = build_scaled(h, h->ilu, dt);
  dev_free(dt, sizeof(double) * (size_t)h->N, h->stream);
  if (st == NDIAG_OK) st = check_status(h);
  h->ilu_mode = st == NDIAG_OK ? mode : -1;
  return st;
}

ndiag_status ssor_apply(ndiag* h, int mode, double omega, const void* r, void* z) {
  if (!h || !r || !z || r == z) return NDIAG_EINVAL;
  if (mode != NDIAG_NATURAL && mode != NDIAG_DECOMPOSED) return NDIAG_EINVAL;
  return do_ssor_apply(h, mode, omega, r, z);
}

ndiag_status ilu0_apply(ndiag* h, const void* r, void* z) {
  if (!h || !r || !z) return NDIAG_EINVAL;
  return do_ilu_apply(h, r, z);
}

ndiag_status ndiag_residual(ndiag* h, const double* b, const double* x, double* r, double* norm2) {
  if (!h || !b || !x || !r) return NDIAG_EINVAL;
  ND_TRY(residual64(h, b, x, r, h->red + SC_R0));
  if (norm2) {
    double v = 0.0;
    ND_CUDA(cudaMemcpyAsync(&v, h->red + SC_R0, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    ND_CUDA(cudaStreamSynchronize(h->stream));
    *norm2 = std::sqrt(v);
  }
  return NDIAG_OK;
}

}  // extern "C"
