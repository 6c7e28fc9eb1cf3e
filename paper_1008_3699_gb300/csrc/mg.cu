// Multigrid V-cycle with the decomposed SSOR sweep as its smoother, as a
// preconditioner of PCG (2D 5-point and 3D 7-point, fp64). The paper names SOR as the usual
// multigrid smoother (Sec. 5); here the decomposed SSOR apply of every level
// is that smoother, the same kernels at each grid size.
//
// Coarse levels are Galerkin products A_c = P^T A P with piecewise-constant
// prolongation P over 2 x 2 (x 2 in 3D) aggregates of cells (the last
// aggregate of an odd side is one cell wide), so every level keeps the 5-point
// (7-point) structure and runs on the library's own sweep path. One V-cycle
// z = B r on level k:
//   z  = S r                            (S: the SSOR apply, symmetric)
//   z += ALPHA P B_{k+1} P^T (r - A z)
//   z += S (r - A z)
// and on the coarsest level KC SSOR-Richardson steps, so B is symmetric for
// PCG. ALPHA over-corrects the piecewise-constant coarse correction, whose
// Galerkin operator is about twice too stiff for smooth error (the usual
// scaling of unsmoothed aggregation: Braess 1995, Notay and Vassilevski 2008).
// B is positive definite when the smoother contracts in the A-norm; with
// subdomains meeting at interior vertices that needs omega < 1 (the coupled
// start-corner blocks give S A the eigenvalue 2 at omega = 1).
#include <cmath>
#include <vector>

#include "blas.h"
#include "internal.h"

namespace nd {

ndiag_status do_ssor_apply(Handle* h, int mode, double omega, const void* r, void* z);
ndiag_status check_device_status(Handle* h);

namespace {

constexpr int KC = 4;          // SSOR-Richardson steps on the coarsest grid
constexpr double ALPHA = 1.8;  // over-correction of the coarse-grid correction
constexpr int64_t NMIN = 32;   // coarsen while either side exceeds this
constexpr int LMAX = 10;       // levels at most
constexpr int NMIN3 = 16;      // 3D: coarsen while a side exceeds this

// r_c = P^T res: each coarse cell sums its (up to) four fine cells, or
// eight in 3D (nz = 1 in 2D), plane by plane in fine-index order
__global__ void restrict_kernel(int nx, int ny, int nz, int nxc, int nyc, int nzc, const double* __restrict__ res,
                                double* __restrict__ rc) {
  const int64_t nc = (int64_t)nxc * nyc * nzc;
  const int64_t pl = (int64_t)nx * ny;
  for (int64_t I = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; I < nc; I += (int64_t)gridDim.x * blockDim.x) {
    const int X = (int)(I % nxc), Y = (int)((I / nxc) % nyc), Z = (int)(I / ((int64_t)nxc * nyc));
    const int x0 = 2 * X, y0 = 2 * Y, z0 = 2 * Z;
    double s = 0.0;
    for (int dz = 0; dz < 2 && z0 + dz < nz; ++dz) {
      const double* q = res + (z0 + dz) * pl;
      const double p0 = q[(int64_t)y0 * nx + x0];
      s = dz == 0 ? p0 : s + p0;
      if (x0 + 1 < nx) s += q[(int64_t)y0 * nx + x0 + 1];
      if (y0 + 1 < ny) {
        s += q[(int64_t)(y0 + 1) * nx + x0];
        if (x0 + 1 < nx) s += q[(int64_t)(y0 + 1) * nx + x0 + 1];
      }
    }
    rc[I] = s;
  }
}
// z += ALPHA P z_c: each fine cell takes its aggregate's value
__global__ void prolong_add_kernel(int nx, int ny, int nz, int nxc, int nyc, const double* __restrict__ zc,
                                   double* __restrict__ z) {
  const int64_t n = (int64_t)nx * ny * nz;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % nx), y = (int)((i / nx) % ny), zz = (int)(i / ((int64_t)nx * ny));
    z[i] += ALPHA * zc[((int64_t)(zz / 2) * nyc + y / 2) * nxc + x / 2];
  }
}
__global__ void add_kernel(int64_t n, double* __restrict__ z, const double* __restrict__ t) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    z[i] += t[i];
}

// Galerkin product P^T A P of a 5-point (2D) or 7-point (3D) matrix
// (diagonal-major, entries P W E S N [B F] as in ndiag_create) over 2 x 2
// (x 2) aggregates, on the host.
std::vector<double> galerkin(const std::vector<double>& A, int s, const int n[3], const int nc[3]) {
  const int64_t N = (int64_t)n[0] * n[1] * n[2], Nc = (int64_t)nc[0] * nc[1] * nc[2];
  std::vector<double> C((size_t)s * Nc, 0.0);
  const int off[6][3] = {{-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};
  for (int z = 0; z < n[2]; ++z)
    for (int y = 0; y < n[1]; ++y)
      for (int x = 0; x < n[0]; ++x) {
        const int64_t i = ((int64_t)z * n[1] + y) * n[0] + x;
        const int X = x / 2, Y = y / 2, Z = z / 2;
        const int64_t I = ((int64_t)Z * nc[1] + Y) * nc[0] + X;
        C[I] += A[i];
        for (int e = 0; e < s - 1; ++e) {
          const int xj = x + off[e][0], yj = y + off[e][1], zj = z + off[e][2];
          if (xj < 0 || xj >= n[0] || yj < 0 || yj >= n[1] || zj < 0 || zj >= n[2]) continue;
          const double a = A[(size_t)(1 + e) * N + i];
          if (xj / 2 == X && yj / 2 == Y && zj / 2 == Z) C[I] += a;  // inside the aggregate
          else C[(size_t)(1 + e) * Nc + I] += a;                     // to the neighbouring aggregate along e
        }
      }
  return C;
}

int grid_for(int64_t n) { return (int)std::min<int64_t>((n + 255) / 256, 4096); }

}  // namespace

struct MgLevel {
  Handle* h = nullptr;  // this level's handle (level 0: the solver's own)
  bool own = false;
  int nx = 0, ny = 0, nz = 1;
  double *r = nullptr, *z = nullptr, *res = nullptr, *t = nullptr;  // device vectors (r, z not on level 0)
  size_t vb = 0;
};

struct Multigrid {
  std::vector<MgLevel> lv;
  double* scratch = nullptr;  // one device scalar (residual norms, unused)
};

void mg_free(Handle* h) {
  if (!h->mg) return;
  Multigrid* M = h->mg;
  for (MgLevel& L : M->lv) {
    for (double* p : {L.r, L.z, L.res, L.t}) dev_free(p, L.vb, h->stream);
    if (L.own) ndiag_destroy(static_cast<ndiag*>(L.h));
  }
  dev_free(M->scratch, sizeof(double), h->stream);
  delete M;
  h->mg = nullptr;
}

namespace {

ndiag_status mg_build(Handle* h) {
  const bool d3 = h->dim == 3;
  if (!((h->dim == 2 && h->stencil == 5) || (d3 && h->stencil == 7)) || h->precision != NDIAG_FP64) {
    set_error("the multigrid preconditioner needs a 2D 5-point or 3D 7-point fp64 handle");
    return NDIAG_EINVAL;
  }
  Multigrid* M = new Multigrid();
  h->mg = M;
  auto vec = [&](MgLevel& L, double*& p) -> bool {
    p = (double*)dev_alloc(L.vb, h->stream);
    return p != nullptr;
  };
  MgLevel L0;
  L0.h = h;
  L0.nx = (int)h->n[0];
  L0.ny = (int)h->n[1];
  L0.nz = d3 ? (int)h->n[2] : 1;
  L0.vb = sizeof(double) * (size_t)h->N;
  M->lv.push_back(L0);
  M->scratch = (double*)dev_alloc(sizeof(double), h->stream);
  if (!M->scratch || !vec(M->lv[0], M->lv[0].res) || !vec(M->lv[0], M->lv[0].t)) return NDIAG_ENOMEM;
  std::vector<double> A((size_t)h->stencil * h->N);
  ND_CUDA(cudaMemcpyAsync(A.data(), h->A64, sizeof(double) * A.size(), cudaMemcpyDeviceToHost, h->stream));
  ND_CUDA(cudaStreamSynchronize(h->stream));
  int n[3] = {L0.nx, L0.ny, L0.nz};
  const int nmin = d3 ? NMIN3 : NMIN;
  while (std::max(n[0], std::max(n[1], n[2])) > nmin && (int)M->lv.size() < LMAX) {
    const int nc[3] = {(n[0] + 1) / 2, (n[1] + 1) / 2, d3 ? (n[2] + 1) / 2 : 1};
    std::vector<double> C = galerkin(A, h->stencil, n, nc);
    MgLevel L;
    L.nx = nc[0];
    L.ny = nc[1];
    L.nz = nc[2];
    L.vb = sizeof(double) * (size_t)nc[0] * nc[1] * nc[2];
    const int64_t n64[3] = {nc[0], nc[1], nc[2]};
    // at least 16 cells a side, at most 16 (2D) or 8 (3D) parts an axis: the
    // sequential path of a coarse sweep stays short while the smoother keeps
    // its quality
    const int pmax = d3 ? 8 : 16;
    const int sub[3] = {std::min(pmax, std::max(1, nc[0] / 16)), std::min(pmax, std::max(1, nc[1] / 16)),
                        d3 ? std::min(pmax, std::max(1, nc[2] / 16)) : 1};
    ndiag* hc = nullptr;
    ND_TRY(ndiag_create(&hc, h->dim, n64, h->stencil, C.data(), sub, NDIAG_FP64, h->stream));
    L.h = hc;
    L.own = true;
    M->lv.push_back(L);
    MgLevel& Lb = M->lv.back();
    if (!vec(Lb, Lb.r) || !vec(Lb, Lb.z) || !vec(Lb, Lb.res) || !vec(Lb, Lb.t)) return NDIAG_ENOMEM;
    A.swap(C);
    for (int a = 0; a < 3; ++a) n[a] = nc[a];
  }
  return NDIAG_OK;
}

ndiag_status vcycle(Multigrid& M, size_t k, double om, const double* r, double* z) {
  MgLevel& L = M.lv[k];
  Handle* hk = L.h;
  const int64_t n = (int64_t)L.nx * L.ny * L.nz;
  const int g = grid_for(n);
  ND_TRY(do_ssor_apply(hk, NDIAG_DECOMPOSED, om, r, z));
  if (k + 1 == M.lv.size()) {
    for (int it = 1; it < KC; ++it) {
      ND_TRY(residual64(hk, r, z, L.res, M.scratch));
      ND_TRY(do_ssor_apply(hk, NDIAG_DECOMPOSED, om, L.res, L.t));
      add_kernel<<<g, 256, 0, hk->stream>>>(n, z, L.t);
      ++hk->launches;
    }
    return NDIAG_OK;
  }
  MgLevel& C = M.lv[k + 1];
  ND_TRY(residual64(hk, r, z, L.res, M.scratch));
  restrict_kernel<<<grid_for((int64_t)C.nx * C.ny * C.nz), 256, 0, hk->stream>>>(L.nx, L.ny, L.nz, C.nx, C.ny, C.nz,
                                                                                 L.res, C.r);
  ++hk->launches;
  ND_CUDA(cudaGetLastError());
  ND_TRY(vcycle(M, k + 1, om, C.r, C.z));
  prolong_add_kernel<<<g, 256, 0, hk->stream>>>(L.nx, L.ny, L.nz, C.nx, C.ny, C.z, z);
  ++hk->launches;
  ND_TRY(residual64(hk, r, z, L.res, M.scratch));
  ND_TRY(do_ssor_apply(hk, NDIAG_DECOMPOSED, om, L.res, L.t));
  add_kernel<<<g, 256, 0, hk->stream>>>(n, z, L.t);
  ++hk->launches;
  ND_CUDA(cudaGetLastError());
  return NDIAG_OK;
}

}  // namespace

// z = B r (one V-cycle), r and z fp64 device vectors of the handle's grid.
// The coarse handles' kernels are counted on the solver's handle.
ndiag_status mg_apply(Handle* h, double omega, const double* r, double* z) {
  if (!h->mg) {
    const ndiag_status st = mg_build(h);
    if (st != NDIAG_OK) {
      mg_free(h);
      return st;
    }
  }
  Multigrid& M = *h->mg;
  int64_t before = 0;
  for (size_t k = 1; k < M.lv.size(); ++k) before += M.lv[k].h->launches;
  const ndiag_status st = vcycle(M, 0, omega, r, z);
  for (size_t k = 1; k < M.lv.size(); ++k) h->launches += M.lv[k].h->launches;
  h->launches -= before;
  return st;
}

ndiag_status mg_check(Handle* h) {
  if (!h->mg) return NDIAG_OK;
  for (size_t k = 1; k < h->mg->lv.size(); ++k) ND_TRY(check_device_status(h->mg->lv[k].h));
  return NDIAG_OK;
}

}  // namespace nd

using namespace nd;

extern "C" ndiag_status mg_apply(ndiag* h, double omega, const double* r, double* z) {
  if (!h || !r || !z) return NDIAG_EINVAL;
  if (!(omega > 0.0 && omega < 2.0)) {
    set_error("the multigrid smoother needs 0 < omega < 2");
    return NDIAG_EINVAL;
  }
  return nd::mg_apply(h, omega, r, z);
}

extern "C" int ndiag_mg_levels(const ndiag* h) { return h && h->mg ? (int)h->mg->lv.size() : 0; }
