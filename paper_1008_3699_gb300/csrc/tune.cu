// Relaxation factor per sweep direction for the stationary decomposed SOR
// iteration. The paper relaxes the two sweep directions of 1D SOR separately
// (omega_L, omega_R; Tables 2-5, over- and under-relaxation with the factors
// searched in [0, 2] to 1e-3) and gives sufficient conditions for convergence
// with different factors (Theorems 1 and 2); this searches the 2^dim factors
// of the decomposed iteration (one per start corner) on the GPU by a
// coordinate search on the number of sweeps to the tolerance.
#include <algorithm>
#include <vector>

#include "internal.h"

extern "C" ndiag_status ndiag_tune_omega(ndiag* h, const double* b, double rtol, int maxit, int budget,
                                         double* omega, int* iters) {
  if (!h || !b || !omega || !iters || !(rtol > 0.0) || maxit < 1 || budget < 1) return NDIAG_EINVAL;
  const int nd_ = 1 << h->dim;
  for (int k = 0; k < nd_; ++k)
    if (!(omega[k] > 0.0 && omega[k] < 2.0)) return NDIAG_EINVAL;
  const size_t bytes = sizeof(double) * (size_t)h->N;
  double* x = (double*)nd::dev_alloc(bytes, h->stream);
  if (!x) return NDIAG_ENOMEM;
  int used = 0;
  ndiag_status err = NDIAG_OK;
  // sweeps to the tolerance from x = 0; maxit + 1 when it does not get there
  auto cost = [&](const std::vector<double>& om) -> int {
    ++used;
    if (cudaMemsetAsync(x, 0, bytes, h->stream) != cudaSuccess) {
      err = NDIAG_EDEVICE;
      return maxit + 1;
    }
    ndiag_solve_info info{};
    const ndiag_status st = krylov_solve(h, NDIAG_STATIONARY, NDIAG_PREC_NONE, NDIAG_DECOMPOSED, om.data(), rtol,
                                         maxit, b, x, &info);
    if (st == NDIAG_OK) return info.iterations;
    if (st != NDIAG_ENOCONV) err = st;
    return maxit + 1;
  };
  std::vector<double> cur(omega, omega + nd_);
  int best = cost(cur);
  double delta = 0.05;
  while (err == NDIAG_OK && delta >= 0.002 && used < budget) {
    bool improved = false;
    for (int k = 0; k < nd_ && used < budget && err == NDIAG_OK; ++k) {
      for (int sgn = 1; sgn >= -1 && used < budget; sgn -= 2) {
        std::vector<double> cand = cur;
        cand[k] = std::min(1.98, std::max(0.02, cur[k] + sgn * delta));
        if (cand[k] == cur[k]) continue;
        const int c = cost(cand);
        if (c < best) {
          best = c;
          cur = cand;
          improved = true;
          break;
        }
      }
    }
    if (!improved) delta *= 0.5;
  }
  nd::dev_free(x, bytes, h->stream);
  if (err != NDIAG_OK) return err;
  std::copy(cur.begin(), cur.end(), omega);
  *iters = best;
  return best <= maxit ? NDIAG_OK : NDIAG_ENOCONV;
}
