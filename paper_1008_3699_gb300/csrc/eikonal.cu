// Decomposed fast sweeping for the eikonal equation |grad u| = f on a 2D grid.
//
// The paper's closing remarks apply its decomposition to the fast sweeping
// method as well. One sweep at phase t: every subdomain runs a Gauss-Seidel
// pass from its start corner (the schedule of the linear sweeps: base corner
// of the phase, flipped along an axis for odd subdomain indices), with Zhao's
// Godunov update (Math. Comp. 74, 2005)
//     a = min(u_W, u_E), b = min(u_S, u_N)         (outside the grid: +inf)
//     |a - b| >= f h :  u~ = min(a, b) + f h
//     otherwise      :  u~ = (a + b + sqrt(2 (f h)^2 - (a - b)^2)) / 2
//     u <- min(u, u~)
// Inside a subdomain, visited cells give new values and the rest old ones;
// cells of other subdomains give old values (the halo of old values of the
// paper's data structure, Sec. 3).
//
// One CTA per subdomain, one thread per row of it, in the frame of the start
// corner. The pass is a wavefront over the anti-diagonals of that frame: at
// diagonal d the thread of row ly updates cell d - ly. Its upstream
// neighbours are its own previous value (left) and the value the thread below
// made at d - 1 (down: a lane shuffle, across warps a shared word, one barrier
// per diagonal); its downstream neighbours and the slowness are old values
// streamed along the row with EK loads in flight. Nothing of the subdomain is
// staged, so many CTAs share an SM. Every operation is
// rounded on its own (no contraction), so a sweep reproduces the plain
// row-by-row pass exactly. The largest change of a sweep goes to a device word
// (atomicMax on the bits of a non-negative double).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>

#include "internal.h"

namespace nd {
namespace {

constexpr int EMAX = 256;  // threads per CTA at most: one per row of the tallest subdomain
constexpr int EK = 4;      // values of each stream in flight per thread

struct EikP {
  int nx, ny;
  Split sx, sy;
  int base;   // start corner of subdomain (0, 0) at this phase
  double h;
  const double* f;
  const double* uo;
  double* un;
  unsigned long long* change;
};

__device__ __forceinline__ double godunov(double a, double b, double fh) {
  const double d = __dsub_rn(a, b);
  if (!(fabs(d) < fh)) return __dadd_rn(fmin(a, b), fh);
  const double q = __dsub_rn(__dmul_rn(2.0, __dmul_rn(fh, fh)), __dmul_rn(d, d));
  return __dmul_rn(__dadd_rn(__dadd_rn(a, b), __dsqrt_rn(q)), 0.5);
}

__global__ void __launch_bounds__(EMAX) eik_sweep_kernel(EikP P) {
  extern __shared__ double hrow[];           // old values of the frame row below row 0
  __shared__ double xfer[2][EMAX / 32];      // last lane's new value, per warp and diagonal parity
  const int ix = blockIdx.x % P.sx.p, iy = blockIdx.x / P.sx.p;
  const int c = P.base ^ (ix & 1) ^ ((iy & 1) << 1);
  const int x0 = P.sx.lo(ix), w = P.sx.len(ix);
  const int y0 = P.sy.lo(iy), hh = P.sy.len(iy);
  const double inf = __longlong_as_double(0x7ff0000000000000LL);
  // frame coordinate -> grid coordinate
  auto gx = [&](int lx) { return (c & 1) ? x0 + w - 1 - lx : x0 + lx; };
  auto gy = [&](int ly) { return (c & 2) ? y0 + hh - 1 - ly : y0 + ly; };
  const int ly = threadIdx.x, lane = ly & 31, wid = ly >> 5;
  const bool row = ly < hh;
  {
    const int Yb = gy(-1);
    const bool ok = Yb >= 0 && Yb < P.ny;
    for (int lx = threadIdx.x; lx < w; lx += blockDim.x)
      hrow[lx] = ok ? __ldcg(P.uo + (int64_t)Yb * P.nx + gx(lx)) : inf;
  }
  // the three streams of this thread's row: old u of the row (frame lx -1..w),
  // old u of the row above (lx 0..w-1) and the slowness (lx 0..w-1)
  const int Yr = gy(row ? ly : 0), Yu = gy(ly + 1);
  const bool up_ok = row && Yu >= 0 && Yu < P.ny;
  const double* urow = P.uo + (int64_t)Yr * P.nx;
  const double* uup = P.uo + (int64_t)(up_ok ? Yu : Yr) * P.nx;
  const double* frow = P.f + (int64_t)Yr * P.nx;
  auto ld_r = [&](int lx) -> double {
    const int X = gx(lx);
    return row && lx >= -1 && lx <= w && X >= 0 && X < P.nx ? __ldcg(urow + X) : inf;
  };
  auto ld_u = [&](int lx) -> double { return up_ok && lx >= 0 && lx < w ? __ldcg(uup + gx(lx)) : inf; };
  auto ld_f = [&](int lx) -> double { return row && lx >= 0 && lx < w ? __ldg(frow + gx(lx)) : 0.0; };
  // slot j of a ring serves the diagonals d = j (mod EK); at diagonal d the
  // thread's cell is lx = d - ly and it needs r(lx + 1), up(lx), f(lx)
  double rr[EK], ru[EK], rf[EK];
#pragma unroll
  for (int j = 0; j < EK; ++j) {
    rr[j] = ld_r(j - ly + 1);
    ru[j] = ld_u(j - ly);
    rf[j] = ld_f(j - ly);
  }
  double left = ld_r(-1);   // new value of the cell to the left (the halo at first)
  double cur = ld_r(-ly);   // old value of the thread's cell
  double v = inf;           // the thread's last new value
  double m = 0.0;
  __syncthreads();
  const int D = w + hh - 1;
  for (int d0 = 0; d0 < D; d0 += EK) {
#pragma unroll
    for (int j = 0; j < EK; ++j) {
      const int d = d0 + j;
      if (d < D) {  // the same for the whole block
        const int lx = d - ly;
        const double right = rr[j], up = ru[j], fc = rf[j];
        rr[j] = ld_r(lx + 1 + EK);
        ru[j] = ld_u(lx + EK);
        rf[j] = ld_f(lx + EK);
        // new value of the cell below, made by the thread below at d - 1
        double down = __shfl_up_sync(0xffffffffu, v, 1);
        if (lane == 0) down = wid == 0 ? (lx >= 0 && lx < w ? hrow[lx] : inf) : xfer[(d - 1) & 1][wid - 1];
        if (row && lx >= 0 && lx < w) {
          const double a = fmin(left, right);
          const double b = fmin(down, up);
          v = fmin(cur, godunov(a, b, __dmul_rn(fc, P.h)));
          if (__double_as_longlong(v) != __double_as_longlong(cur)) m = fmax(m, __dsub_rn(cur, v));
          P.un[(int64_t)Yr * P.nx + gx(lx)] = v;
          left = v;
        }
        cur = right;
        if (lane == 31) xfer[d & 1][wid] = v;
        __syncthreads();
      }
    }
  }
  // largest change of the CTA
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0 && m > 0.0) atomicMax(P.change, (unsigned long long)__double_as_longlong(m));
}

bool device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace
}  // namespace nd

using namespace nd;

struct ndiag_eik {
  int nx = 0, ny = 0;
  Split sx{}, sy{};
  double h = 0.0;
  cudaStream_t stream = nullptr;
  double* f = nullptr;
  double* buf = nullptr;  // two vectors for the solve
  size_t buf_bytes = 0;
  unsigned long long* change = nullptr;
  unsigned long long* change_host = nullptr;
  int threads = 0;
  size_t smem = 0;
  int64_t launches = 0;
};

namespace {

ndiag_status eik_launch(ndiag_eik* e, int64_t t, const double* uo, double* un) {
  EikP P;
  P.nx = e->nx;
  P.ny = e->ny;
  P.sx = e->sx;
  P.sy = e->sy;
  P.base = base_corner(2, t);
  P.h = e->h;
  P.f = e->f;
  P.uo = uo;
  P.un = un;
  P.change = e->change;
  ++e->launches;
  eik_sweep_kernel<<<e->sx.p * e->sy.p, e->threads, e->smem, e->stream>>>(P);
  ND_CUDA(cudaGetLastError());
  return NDIAG_OK;
}

ndiag_status read_change(ndiag_eik* e, double* out) {
  ND_CUDA(cudaMemcpyAsync(e->change_host, e->change, sizeof(unsigned long long), cudaMemcpyDeviceToHost, e->stream));
  ND_CUDA(cudaStreamSynchronize(e->stream));
  const unsigned long long bits = *e->change_host;
  std::memcpy(out, &bits, sizeof(double));
  return NDIAG_OK;
}

}  // namespace

extern "C" {

ndiag_status eikonal_create(ndiag_eik** out, const int64_t n[2], double h, const double* f, const int sub[2],
                            void* cuda_stream) {
  if (!out) return NDIAG_EINVAL;
  *out = nullptr;
  if (!n || !f || !sub || !(h > 0.0)) return NDIAG_EINVAL;
  if (n[0] < 1 || n[1] < 1 || n[0] > (1 << 20) || n[1] > (1 << 20) || sub[0] < 1 || sub[1] < 1 ||
      sub[0] > n[0] || sub[1] > n[1]) {
    set_error("eikonal_create: bad sizes or subdomains");
    return NDIAG_EINVAL;
  }
  const int64_t N = n[0] * n[1];
  for (int64_t i = 0; i < N; ++i)
    if (!(f[i] >= 0.0) || std::isinf(f[i])) {
      set_error("eikonal_create: slowness must be finite and >= 0");
      return NDIAG_EINVAL;
    }
  ndiag_eik* e = new ndiag_eik();
  e->nx = (int)n[0];
  e->ny = (int)n[1];
  e->sx = Split{sub[0], e->nx / sub[0], e->nx % sub[0]};
  e->sy = Split{sub[1], e->ny / sub[1], e->ny % sub[1]};
  e->h = h;
  e->stream = (cudaStream_t)cuda_stream;
  const int wmax = e->sx.q + (e->sx.r ? 1 : 0), hmax = e->sy.q + (e->sy.r ? 1 : 0);
  e->smem = sizeof(double) * (size_t)wmax;
  e->threads = 32 * ((hmax + 31) / 32);
  if (e->smem > 200 * 1024 || hmax > EMAX) {
    delete e;
    set_error("eikonal_create: a subdomain may have at most 256 rows and 25600 columns");
    return NDIAG_EINVAL;
  }
  // the same ceiling for every handle, so that handles of different widths coexist
  if (cudaFuncSetAttribute(eik_sweep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) !=
      cudaSuccess) {
    cudaGetLastError();
    delete e;
    set_error("eikonal_create: shared memory attribute refused");
    return NDIAG_EDEVICE;
  }
  e->f = (double*)dev_alloc(sizeof(double) * (size_t)N, e->stream);
  e->change = (unsigned long long*)dev_alloc(sizeof(unsigned long long), e->stream);
  if (!e->f || !e->change || cudaMallocHost(&e->change_host, sizeof(unsigned long long)) != cudaSuccess) {
    cudaGetLastError();
    eikonal_destroy(e);
    return NDIAG_ENOMEM;
  }
  if (cudaMemcpyAsync(e->f, f, sizeof(double) * (size_t)N, cudaMemcpyHostToDevice, e->stream) != cudaSuccess ||
      cudaStreamSynchronize(e->stream) != cudaSuccess) {
    eikonal_destroy(e);
    return cuda_status(cudaGetLastError(), "eikonal_create copy");
  }
  *out = e;
  return NDIAG_OK;
}

void eikonal_destroy(ndiag_eik* e) {
  if (!e) return;
  dev_free(e->f, 0, e->stream);
  dev_free(e->buf, e->buf_bytes, e->stream);
  dev_free(e->change, sizeof(unsigned long long), e->stream);
  cudaStreamSynchronize(e->stream);
  if (e->change_host) cudaFreeHost(e->change_host);
  delete e;
}

ndiag_status eikonal_sweep(ndiag_eik* e, int64_t t, const double* u_old, double* u_new, double* change) {
  if (!e || !u_old || !u_new || u_old == u_new) return NDIAG_EINVAL;
  ND_CUDA(cudaMemsetAsync(e->change, 0, sizeof(unsigned long long), e->stream));
  ND_TRY(eik_launch(e, t, u_old, u_new));
  if (change) return read_change(e, change);
  return NDIAG_OK;
}

ndiag_status eikonal_solve(ndiag_eik* e, double* u, double delta, int max_rounds, ndiag_eik_info* info) {
  const auto t0 = std::chrono::steady_clock::now();
  if (!e || !u || !(delta >= 0.0) || max_rounds < 1) return NDIAG_EINVAL;
  const size_t vb = sizeof(double) * (size_t)e->nx * (size_t)e->ny;
  const bool dev_u = device_ptr(u);
  if (e->buf_bytes < 2 * vb) {
    dev_free(e->buf, e->buf_bytes, e->stream);
    e->buf = (double*)dev_alloc(2 * vb, e->stream);
    e->buf_bytes = e->buf ? 2 * vb : 0;
    if (!e->buf) return NDIAG_ENOMEM;
  }
  double* a = e->buf;
  double* b = e->buf + vb / sizeof(double);
  ND_CUDA(cudaMemcpyAsync(a, u, vb, dev_u ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, e->stream));
  int64_t t = 0;
  double m = 0.0;
  bool done = false;
  for (int r = 0; r < max_rounds && !done; ++r) {
    ND_CUDA(cudaMemsetAsync(e->change, 0, sizeof(unsigned long long), e->stream));
    for (int k = 0; k < 4; ++k, ++t) {
      ND_TRY(eik_launch(e, t, a, b));
      std::swap(a, b);
    }
    ND_TRY(read_change(e, &m));
    done = m <= delta;
  }
  ND_CUDA(cudaMemcpyAsync(u, a, vb, dev_u ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, e->stream));
  ND_CUDA(cudaStreamSynchronize(e->stream));
  if (info) {
    info->sweeps = (int)t;
    info->converged = done ? 1 : 0;
    info->change = m;
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    info->launches = e->launches;
  }
  return done ? NDIAG_OK : NDIAG_ENOCONV;
}

}  // extern "C"
