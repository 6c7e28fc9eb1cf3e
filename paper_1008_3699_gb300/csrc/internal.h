// Internal declarations of the GB300 sweep library (not part of the C ABI).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/ndiag.h"

namespace nd {

// ---------------------------------------------------------------------------
// Errors and allocation
// ---------------------------------------------------------------------------
void set_error(const std::string& msg);
ndiag_status cuda_status(cudaError_t e, const char* what);
#define ND_CUDA(call)                                              \
  do {                                                             \
    cudaError_t e_ = (call);                                       \
    if (e_ != cudaSuccess) return ::nd::cuda_status(e_, #call);    \
  } while (0)
#define ND_TRY(call)                              \
  do {                                            \
    ndiag_status s_ = (call);                     \
    if (s_ != NDIAG_OK) return s_;                \
  } while (0)

void* dev_alloc(size_t bytes, cudaStream_t s);
// Threads of the server allocate with cudaMallocAsync even when hooks are set.
void use_plain_allocator_on_this_thread(bool on);
void dev_free(void* p, size_t bytes, cudaStream_t s);

// Stencil entries (diagonal-major storage order of the C ABI).
enum { EC = 0, EW = 1, EE = 2, ES = 3, EN = 4, EB = 5, EF = 6,
       ESW = 5, ESE = 6, ENW = 7, ENE = 8 };

// Internal ordering value: the natural ordering run backwards (the backward
// halves of ILU(0) and SSOR in natural mode).
enum { MODE_NATURAL_REV = 2 };

// Sweep kinds (what one cell update computes; see sweep2d.cu).
enum SweepKind {
  KIND_SOR = 0,         // x = (1-w) u + w (inv*b - sum_old c u) - w sum_J c x
  KIND_TRI_SCALED = 1,  // x = inv*r - w sum_J c x     (ILU forward, SSOR forward)
  KIND_TRI_UNIT = 2     // x = r - w sum_J c x         (ILU backward)
};

// Scaled coefficient set: inv[i] = 1/pivot_i, c[e][i] = A(i, e) / pivot_i for
// every off-diagonal entry e (pivot = a_ii for SOR/SSOR, d~_i for ILU(0)).
struct ScaledSet {
  void* base = nullptr;  // one allocation: s arrays of N values (inv, then entries 1..s-1)
  size_t bytes = 0;
  unsigned version = 0;  // bumped whenever the values change (invalidates line tables)
  // 3D: the same arrays in level order (built on first use by the pencil sweeps)
  void* lev = nullptr;
  size_t lev_bytes = 0;
  unsigned lev_version = ~0u;
};

// Coefficients of the coupled start lines of one sweep phase (2D): for every
// subdomain with a coupled start row / column and every position along it,
// the pair terms of Eq. 2d:sor2b2 that do not depend on the right-hand side.
struct LineTable {
  const void* set_base = nullptr;
  unsigned set_version = 0;
  int base = -1;          // start corner of subdomain 0
  int om1 = 1;
  double om[4] = {1, 1, 1, 1};
  void* buf = nullptr;
  size_t bytes = 0;
};


// Device-side status words (error flag written by bounded waits).
struct DevStatus {
  int timeout;      // a bounded wait gave up
  int zero_pivot;   // ILU factor met a zero pivot
};

struct Workspace {
  void* p = nullptr;
  size_t bytes = 0;
};

struct ProfRec {
  cudaEvent_t a = nullptr, b = nullptr;
  double bytes = 0.0;
};

struct Multigrid;  // mg.cu

// A kernel's private copy of a scaled set in its own operand order (the
// 9-point wavefront sweeps, sweep9w.cu; the 3D forward block records,
// sweep3d.cu): one per phase and kind, rebuilt when the set or the partition
// changes.
struct PackCache {
  const void* set_base = nullptr;
  unsigned set_version = 0;
  int64_t t = -1;
  int kind = -1;
  int sub0 = 0, sub1 = 0;
  double* buf = nullptr;
  size_t bytes = 0;
  double* rdx = nullptr;
  size_t rdx_bytes = 0;
};

struct Handle {
  int dim = 0, stencil = 0, precision = 0;
  int64_t n[3] = {1, 1, 1};
  int64_t N = 0;
  int sub[3] = {1, 1, 1};
  cudaStream_t stream = nullptr;
  int sm_count = 0;
  size_t vec_bytes = 0;   // bytes of one vector in the handle's precision

  double* A64 = nullptr;  // s * N raw matrix, fp64 (residuals, SpMV)
  void* Alo = nullptr;    // s * N raw matrix in the sweep precision (fp32 inner SpMV)
  ScaledSet sor;          // pivots a_ii
  ScaledSet ilu;          // pivots d~_i
  ScaledSet sorT;         // transposed entries A(j, i) / a_ii (SSOR backward solve)
  unsigned* vcount = nullptr;    // per subdomain vertex: edges finished (self-resetting)
  size_t vcount_bytes = 0;
  int ilu_mode = -1;

  // sweep scratch: progress flags / ticket / twin handoff for multi-CTA subdomains
  unsigned* sync = nullptr;
  size_t sync_bytes = 0;
  void* twin_hand = nullptr;
  size_t twin_hand_bytes = 0;
  std::vector<LineTable> line_tables;  // per (coefficient set, phase, relaxation)
  DevStatus* status = nullptr;   // device

  // Krylov workspace (allocated on first use)
  Workspace kws;
  double* red = nullptr;         // reduction partials + results (device)
  size_t red_bytes = 0;
  double* red_host = nullptr;    // pinned mirror of the results
  void* tmp = nullptr;           // one vector in sweep precision (ssor/ilu intermediates)
  size_t tmp_bytes = 0;
  // per-iteration record of the fp64 Krylov solves (ndiag_set_history)
  double* hist_dev = nullptr;    // device, 4 values per iteration
  int hist_cap = 0;              // iterations it holds
  double* hist_user = nullptr;   // host buffer the caller gave

  // counters (ndiag_profile / ndiag_read_counters)
  int64_t launches = 0;
  int64_t sweep_launches = 0;
  double sweep_ms = 0.0;
  double sweep_bytes = 0.0;
  bool profiling = false;
  std::vector<ProfRec> prof;
  std::vector<cudaEvent_t> ev_pool;
  Multigrid* mg = nullptr;       // V-cycle hierarchy (built on the first multigrid apply)
  std::vector<PackCache> w9pack; // 9-point wavefront operands (sweep9w.cu)
  std::vector<PackCache> brec3d; // 3D forward block records (sweep3d.cu)
  bool w9_wave = true;           // 9-point wavefront sweeps where they apply
  bool w3_wave = true;           // 3D wavefront pencil walks where they apply
};

// Sweep-launch timing: brackets a sweep kernel with events when profiling is
// on and records its algorithmic bytes.
int prof_begin(Handle* h);
void prof_end(Handle* h, int slot, double bytes);

// Partition of n cells into p parts, the first n mod p parts one longer.
struct Split {
  int p, q, r;
  __host__ __device__ int lo(int k) const { return k * q + (k < r ? k : r); }
  __host__ __device__ int len(int k) const { return q + (k < r ? 1 : 0); }
};
// 9-point sweeps (sweep9.cu): whether subdomains of this height need all CTAs
// resident (their x-interfaces advance in step through global memory)
bool sweep9_needs_residency(int64_t ny, int py);
// part holding coordinate x
__host__ __device__ inline int split_find(const Split& s, int x) {
  const int big = s.r * (s.q + 1);
  return x < big ? x / (s.q + 1) : s.r + (x - big) / s.q;
}

// Start corner of subdomain 0 at phase t (Sec. 2 step (ii); Sec. 3 "Sweeping
// directions"; Sec. 4): 1D alternates starting left-to-right; in 2D/3D the
// corner is the all-ones corner with floor((t mod 2^d)/2) flipped on x, y, and
// reversed on odd t.
int base_corner(int dim, int64_t t);
// Forward phase of the preconditioners: subdomain 0 sweeps from its origin.
inline int64_t fwd_phase(int dim) { return dim == 1 ? 0 : 1; }

// Launchers (sweep2d.cu)
ndiag_status launch_sweep2d(Handle* h, int kind, int mode, int64_t t, const double* omega,
                            const ScaledSet& set, const void* rhs, const void* xold, void* xnew);
ndiag_status launch_sweep2d_ex(Handle* h, int kind, int mode, int64_t t, const double* omega,
                               const ScaledSet& set, const void* rhs, const void* xold, void* xnew,
                               double beta_scale, bool reverse_interior);
ndiag_status launch_ssor_edges2d(Handle* h, int mode, double omega, const void* w, void* z);
// staged kernel (sweep2d_staged.cu); NDIAG_EINVAL when it does not cover the request
ndiag_status launch_sweep2d_staged(Handle* h, int kind, int mode, int64_t t, const double* omega,
                                   const ScaledSet& set, const void* rhs, const void* xold, void* xnew,
                                   double beta_scale, bool rev);
ndiag_status launch_tri_sweep2d_scratch(Handle* h, int kind, int mode, int64_t t, const ScaledSet& set,
                                        const void* rhs, void* xnew, unsigned* sync, size_t sync_bytes,
                                        void* twin, size_t twin_bytes);
ndiag_status build_scaled(Handle* h, ScaledSet& set, const double* piv);
// the same from another s x N matrix A (entries / piv, 1 / piv)
ndiag_status build_scaled_from(Handle* h, ScaledSet& set, const double* A, const double* piv);
// natural-order ILU(0) of a 9-point matrix into F (9 x N, ilu9n.cu)
ndiag_status launch_ilu_factor9_natural(Handle* h, double* F);
// decomposed full ILU(0) of a 9-point matrix into F (9 x N, ilu9n.cu): the
// IKJ elimination of every subdomain's block in its forward-sweep order
ndiag_status launch_ilu_factor9_full(Handle* h, double* F);
// One prepared launch of the staged 2D sweep over several handles (a batch of
// independent problems): device arrays of per-problem parameters and slab
// offsets, rebuilt by batch_sweep_prepare, launched by batch_sweep_launch
// (graph-capturable: no host work).
struct BatchSweep {
  int precision = 0, kind = 0, np = 0;
  bool om1 = true;
  unsigned total = 0;  // slabs (CTAs) of the launch
  double bytes = 0.0;  // algorithmic bytes of one launch
  void* params = nullptr;
  size_t params_bytes = 0;
  unsigned* off = nullptr;
  size_t off_bytes = 0;
  std::vector<unsigned char> host_params;
  std::vector<unsigned> host_off;
};
// set_sel: 0 SOR set, 1 ILU(0) set, 2 transposed SOR set
ndiag_status batch_sweep_prepare(BatchSweep& b, Handle* const* hs, int np, int kind, int mode, int64_t t,
                                 const double* omega, int set_sel, const void* const* rhs, const void* const* xold,
                                 void* const* xnew, double beta_scale, bool rev, cudaStream_t s);
ndiag_status batch_sweep_launch(const BatchSweep& b, cudaStream_t s);
void batch_sweep_free(BatchSweep& b, cudaStream_t s);
// the SSOR interface chains of several handles in one launch (ssor2d.cu)
ndiag_status batch_edges_prepare(BatchSweep& b, Handle* const* hs, int np, double omega, const void* const* w,
                                 void* const* z, cudaStream_t s);
ndiag_status batch_edges_launch(const BatchSweep& b, cudaStream_t s);

// Device status of a handle, read after a batch of launches (api.cu)
ndiag_status check_device_status(Handle* h);
// Re-partition a handle into sub[] subdomains (batch.cu, the autotuner)
void handle_set_sub(Handle* h, const int sub[3]);

// 3D 7-point sweeps by levels (sweep3d.cu); `transposed` solves (D + w L^T) y = v
ndiag_status launch_sweep3d(Handle* h, int kind, int mode, int64_t t, const double* omega, const ScaledSet& set,
                            const void* rhs, const void* xold, void* xnew, double beta_scale, bool transposed);
ndiag_status launch_ilu_factor3d_into(Handle* h, int mode, double* out);
// 2D 9-point sweeps by levels (sweep9.cu); D-ILU pivots of the decomposed 9-point factor
ndiag_status launch_sweep9(Handle* h, int kind, int mode, int64_t t, const double* omega, const ScaledSet& set,
                           const void* rhs, const void* xold, void* xnew, double beta_scale);
ndiag_status launch_ilu_factor9_into(Handle* h, int mode, double* out);
// fp64 decomposed 9-point triangular sweeps as a warp-synchronous wavefront
// (sweep9w.cu); NDIAG_EINVAL, with nothing launched, outside its cover
ndiag_status launch_sweep9w(Handle* h, int kind, int mode, int64_t t, const ScaledSet& set, const void* rhs,
                            void* xnew);
void w9pack_free(Handle* h);  // frees the 9-point operand copies and the 3D block records
ndiag_status build_scaled_transposed(Handle* h, ScaledSet& set);

// BLAS-1 and SpMV (blas.cu)
ndiag_status spmv64(Handle* h, const double* x, double* y);
ndiag_status residual64(Handle* h, const double* b, const double* x, double* r, double* norm2_dev);
int reduce_blocks(const Handle* h);

// Multigrid V-cycle preconditioner (mg.cu): z = B r on a 2D 5-point fp64
// handle; the hierarchy is built on the first call and freed by mg_free.
ndiag_status mg_apply(Handle* h, double omega, const double* r, double* z);
ndiag_status mg_check(Handle* h);  // device status of the coarse levels
void mg_free(Handle* h);

}  // namespace nd

struct ndiag : nd::Handle {};
