// Vector kernels used by the Krylov drivers (blas.cu).
#pragma once
#include "internal.h"

namespace nd {

// Reduction target: block partials, a self-resetting arrival counter, and
// where the last block writes the final sums.
struct Reduce {
  double* part = nullptr;
  unsigned* counter = nullptr;
  double* res = nullptr;
};

// Layout of Handle::red (doubles): [0, 8) arrival counters, [SC_BASE, RED_RES)
// device scalars of the Krylov drivers, then RED_SLOTS regions of partials.
enum { RED_SLOTS = 4, RED_RES = 64 };
enum {
  SC_BASE = 16,
  SC_RHO = SC_BASE, SC_RHO_OLD, SC_ALPHA, SC_OM, SC_RV, SC_TS, SC_TT, SC_SS, SC_RR, SC_RHO_NEXT,
  SC_RZ, SC_RZ_NEW, SC_PQ, SC_BB, SC_R0, SC_TOL2,
  // device-resident iteration: state word, iterations done, limit, tolerance
  SC_DONE, SC_ITER, SC_MAXIT, SC_TOL, SC_END
};
// SC_DONE values: the iteration runs (0) or has stopped, and why. Once it is
// non-zero the update kernels leave x, r, p and the scalars as they are.
enum { DONE_RUN = 0, DONE_CONV = 1, DONE_BREAK = 2, DONE_BREAK_NONFINITE = 3, DONE_BREAK_OMEGA = 4,
       DONE_MAXIT = 5 };

int grid_blocks(const Handle* h);
size_t reduce_bytes(const Handle* h);
Reduce reduce_slot(Handle* h, int slot);

ndiag_status spmv64(Handle* h, const double* x, double* y);
template <class T> ndiag_status spmv_any(Handle* h, const T* x, T* y);
// y = A x and res[0] = (w, y); if two: res[1] = (y, y)
template <class T> ndiag_status spmv_dot(Handle* h, const T* x, T* y, const T* w, double* res, int slot,
                                         bool two = false);
ndiag_status residual64(Handle* h, const double* b, const double* x, double* r, double* res);
ndiag_status residual64_to32(Handle* h, const double* b, const double* x, float* r, double* res);
template <class T> ndiag_status dots(Handle* h, int nv, const T* a0, const T* b0, const T* a1, const T* b1,
                                     const T* a2, const T* b2, double* res, int slot);
// with inv and sp / ss: also sp = inv .* p, ss = inv .* s (pre-scaled sweep input)
template <class T> ndiag_status bicg_p(Handle* h, const T* r, T* p, const T* v, const double* sc, int first,
                                       const T* inv = nullptr, T* sp = nullptr);
template <class T> ndiag_status bicg_s(Handle* h, const T* r, const T* v, T* s, double* sc,
                                       const T* inv = nullptr, T* ss = nullptr);
template <class T> ndiag_status bicg_xr(Handle* h, T* x, const T* ph, const T* sh, T* r, const T* s,
                                        const T* t, const T* rh, double* sc);
template <class T> ndiag_status axpy_alpha(Handle* h, T* x, const T* ph, const double* sc);
template <class T> ndiag_status cg_xr(Handle* h, T* x, const T* p, T* r, const T* q, double* sc);
template <class T> ndiag_status cg_p(Handle* h, const T* z, T* p, const double* sc, int first);
template <class T> ndiag_status scale(Handle* h, T* x, double f);
template <class T> ndiag_status mul_diag(Handle* h, const T* x, T* y);
// sc[dst] = sc[src] unless the iteration has stopped (sc[SC_DONE] != 0)
ndiag_status copy_scalar(Handle* h, double* sc, int dst, int src);
ndiag_status to32(Handle* h, const double* s, float* d);
ndiag_status add_to(Handle* h, double* x, const float* e);

}  // namespace nd
