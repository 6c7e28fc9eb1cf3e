/*
 * ndiag.h -- C ABI of the GB300 library for the decomposed ("parallel")
 * sequential sweep on structured n-diagonal matrices:
 *   R. Tavakoli, "Parallelizing sequential sweeping on structured grids --
 *   fully parallel SOR/ILU preconditioners for structured n-diagonal
 *   matrices", arXiv 1008.3699.
 *
 * Conventions (all entry points):
 *  - Every call returns an ndiag_status and never aborts. NDIAG_OK = 0.
 *  - Constructors (ndiag_create, ndiag_batch_create, ndiag_server_create,
 *    eikonal_create) set *out to NULL first, so it is NULL after any failure.
 *  - Vectors are in natural cell order (x fastest, then y, then z).
 *  - "device" pointers are CUDA device pointers on the handle's device, owned
 *    by the caller; the library neither frees nor retains them after the call.
 *  - The library owns what it copies at create time (diagonals, scaled
 *    coefficients, factors, the partition and schedule tables) and its Krylov
 *    workspaces; ndiag_destroy releases them.
 *  - Calls are ordered on the handle's CUDA stream. Calls that return values
 *    to the host (krylov_solve, ndiag_residual_norm) synchronise that stream.
 *    A device-side failure (a bounded wait that timed out) is reported at the
 *    next synchronising call as NDIAG_ETIMEOUT.
 *  - Not thread-safe per handle; distinct handles may be used concurrently.
 *
 * Matrix storage (Eq. d2d; Def. "structured n-diagonal matrix", Sec. 7): a
 * structured n-diagonal matrix is given diagonal-major, s arrays of N values,
 * entry k of row i being A(i, i + off_k) in the stencil order
 *     5-point (2D): C W E S N
 *     7-point (3D): C W E S N B F
 *     9-point (2D): C W E S N SW SE NW NE
 * Entries that point outside the grid must be 0 (Dirichlet values are folded
 * into the right-hand side, Eq. 1d:mat).
 */
#ifndef NDIAG_H
#define NDIAG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ndiag ndiag;

typedef enum {
  NDIAG_OK = 0,
  NDIAG_EINVAL = 1,     /* bad argument (size, pointer, enum, unsupported stencil) */
  NDIAG_ENOMEM = 2,     /* device or host allocation failed */
  NDIAG_ENOCONV = 3,    /* iteration limit reached before the tolerance */
  NDIAG_EBREAKDOWN = 4, /* Krylov breakdown (rho = 0, (p,Ap) = 0, ...) or zero pivot */
  NDIAG_EDEVICE = 5,    /* CUDA error; the message is in ndiag_last_error() */
  NDIAG_ETIMEOUT = 6,   /* a bounded device-side wait gave up */
  NDIAG_EBUSY = 7,      /* serving: request not finished yet */
  NDIAG_ESTATE = 8      /* call out of order (e.g. ilu0_apply before ilu0_factor) */
} ndiag_status;

/* Precision of the sweeps and of the stored coefficients. */
enum {
  NDIAG_FP64 = 0,     /* fp64 vectors and coefficients */
  NDIAG_FP32 = 1,     /* fp32 vectors and coefficients */
  NDIAG_FP32_D16 = 2  /* fp32 vectors, coefficients stored as fp16 */
};

/* Ordering of a sweep. */
enum {
  NDIAG_NATURAL = 0,    /* lexicographic order over the whole grid */
  NDIAG_DECOMPOSED = 1, /* the paper's decomposed multi-frontal order */
  /* ilu0_factor only: the decomposed order with the full ILU(0) of every
   * subdomain's block (modified off-diagonals on the 9-point molecule) */
  NDIAG_DECOMPOSED_FULL = 3
};

enum { NDIAG_PCG = 0, NDIAG_BICGSTAB = 1, NDIAG_STATIONARY = 2 };
enum { NDIAG_PREC_NONE = 0, NDIAG_PREC_SSOR = 1, NDIAG_PREC_ILU0 = 2, NDIAG_PREC_MG = 3 };

/* Optional device allocator (e.g. a framework's caching allocator). Without
 * one the library calls cudaMallocAsync / cudaFreeAsync on its stream. */
typedef void* (*ndiag_alloc_fn)(size_t bytes, void* cuda_stream, void* ctx);
typedef void (*ndiag_free_fn)(void* ptr, size_t bytes, void* cuda_stream, void* ctx);
ndiag_status ndiag_set_allocator(ndiag_alloc_fn alloc, ndiag_free_fn release, void* ctx);

/* Text of the last error seen by this thread ("" if none). */
const char* ndiag_last_error(void);

/*
 * ndiag_create -- copy a structured n-diagonal matrix to the device and build
 * the partition and sweep schedule.
 *   dim       2 or 3.
 *   n         cells per axis, n[2] ignored when dim = 2; 1 <= n[a] <= 2^20 and
 *             N = the product of the n[a] below 2^31.
 *   stencil   5 (dim 2), 7 (dim 3) or 9 (dim 2).
 *   diags     HOST array, stencil * N doubles, diagonal-major (see above);
 *             read during the call only (the caller keeps ownership).
 *   sub       subdomains per axis (Sec. 3 "Domain decomposition"): a Cartesian
 *             split into nearly equal parts, the first n mod p parts one cell
 *             longer; 1 <= sub[a] <= n[a].
 *   precision NDIAG_FP64, NDIAG_FP32 or NDIAG_FP32_D16 (the precision of the
 *             sweeps; residuals, dots and norms are always fp64).
 *   cuda_stream  cudaStream_t (NULL = legacy default stream).
 * Errors: NDIAG_EINVAL (a null pointer, dim/stencil, sizes, subdomain counts,
 * precision, a diagonal entry that is not > 0, NaN included), NDIAG_ENOMEM,
 * NDIAG_EDEVICE (no usable CUDA device).
 */
ndiag_status ndiag_create(ndiag** out, int dim, const int64_t n[3], int stencil,
                          const double* diags, const int sub[3], int precision,
                          void* cuda_stream);

void ndiag_destroy(ndiag* h);

/* Number of cells N and the handle's precision. */
int64_t ndiag_cells(const ndiag* h);
int ndiag_precision(const ndiag* h);

/*
 * sor_sweep -- one SOR sweep u^(k) -> u^(k+1) at schedule phase t
 * (Eqs. sor2d_sw..sor2d_nw; coupled start nodes by Eqs. 2d:sor4b4 and
 * 2d:sor2b2; 3D by Sec. 4; the splitting form of Eq. ca2d:matiter):
 *     (D + w L_J) u+ = ((1 - w) D - w U_J) u + w b,
 * J = the implicit set of phase t, w = omega[start corner of the row's
 * subdomain] (corner bit a set when the subdomain starts at its maximum
 * coordinate along axis a; 2^dim entries, HOST array).
 *   mode   NDIAG_DECOMPOSED (paper) or NDIAG_NATURAL (lexicographic).
 *   b, x_old, x_new  DEVICE vectors of N values in the handle's precision
 *          (double for FP64, float otherwise). x_new must not alias x_old:
 *          a sweep reads old values of neighbouring subdomains (the halo of
 *          Sec. 3 "Data structure") while they are being overwritten.
 * Asynchronous on the handle's stream. Errors: NDIAG_EINVAL (a null pointer,
 * x_new == x_old, unknown mode), NDIAG_EDEVICE.
 */
ndiag_status sor_sweep(ndiag* h, int mode, const double* omega, int64_t t, const void* b,
                       const void* x_old, void* x_new);

/*
 * ssor_apply -- symmetric SSOR preconditioner (Sec. 2: SSOR = a sweep and its
 * reverse; Sec. 5), in the SPD form usable inside CG:
 *     z = w (2 - w) (D + w L_J^T)^-1 D (D + w L_J)^-1 r,
 * J = implicit set of the forward phase (the phase at which subdomain 0
 * sweeps from the origin corner; with one subdomain this is classical SSOR).
 *   r, z  DEVICE vectors (handle precision), z must not alias r.
 * Asynchronous on the handle's stream. Errors: NDIAG_EINVAL (a null pointer,
 * z == r, unknown mode, omega outside (0, 2), a 9-point handle: its
 * transposed sweep is not provided), NDIAG_EDEVICE.
 */
ndiag_status ssor_apply(ndiag* h, int mode, double omega, const void* r, void* z);

/*
 * mg_apply -- one multigrid V-cycle z = B r with the decomposed SSOR apply as
 * smoother on every level (the sweep used as a multigrid smoother, Sec. 5,
 * opening paragraph), the preconditioner that krylov_solve runs for
 * NDIAG_PREC_MG. On level k (level 0 = this handle):
 *     z  = S_k r
 *     z += 1.8 P_k B_{k+1} P_k^T (r - A_k z)
 *     z += S_k (r - A_k z)
 * S_k = ssor_apply(DECOMPOSED, omega) of level k; P_k = piecewise-constant
 * prolongation over 2 x 2 cell aggregates (x // 2, y // 2), in 3D 2 x 2 x 2
 * (z // 2 as well); A_{k+1} = P_k^T A_k P_k (5-point / 7-point again), split
 * into min(16, max(1, n / 16)) parts per axis (3D: min(8, max(1, n / 16)));
 * coarsening stops when every side is <= 32 cells (3D: 16) or at 10 levels;
 * the coarsest level takes 4 steps of SSOR-Richardson. B is symmetric;
 * it is positive definite when S contracts in the A-norm, which for subdomains
 * meeting at interior vertices needs omega < 1.
 *   r, z  fp64 DEVICE vectors of N values, z must not alias r.
 * The first call builds the hierarchy on the host from the handle's matrix
 * (a blocking device-to-host copy), later calls are asynchronous.
 * Errors: NDIAG_EINVAL (not a 2D 5-point or 3D 7-point fp64 handle, omega
 * outside (0, 2)), NDIAG_ENOMEM.
 */
ndiag_status mg_apply(ndiag* h, double omega, const double* r, double* z);

/* Levels of the handle's multigrid hierarchy (0 before the first MG use). */
int ndiag_mg_levels(const ndiag* h);

/*
 * ndiag_selftest_wait -- exercises the failure path of the bounded
 * device-side waits that the sweeps use between CTAs: one warp waits on a
 * device word that nothing sets, gives up after the bound (about 2 s of GPU
 * clock), records the timeout and returns. Returns NDIAG_ETIMEOUT when the
 * path works (the status word is cleared again and the handle stays usable);
 * NDIAG_OK would mean the wait did not run out.
 */
ndiag_status ndiag_selftest_wait(ndiag* h);

/*
 * Fast sweeping for the eikonal equation |grad u| = f on an nx x ny grid of
 * spacing h, decomposed like the linear sweeps (the paper's closing remarks
 * apply its decomposition to the fast sweeping method). One sweep at phase t:
 * every subdomain runs a Gauss-Seidel pass from its start corner (the same
 * schedule as sor_sweep), with the Godunov update of Zhao's fast sweeping
 * method (Math. Comp. 74, 2005):
 *     a = min(u_W, u_E), b = min(u_S, u_N)          (outside the grid: +inf)
 *     |a - b| >= f h :  u~ = min(a, b) + f h
 *     otherwise      :  u~ = (a + b + sqrt(2 (f h)^2 - (a - b)^2)) / 2
 *     u <- min(u, u~)
 * Inside a subdomain visited cells give new values and the others old ones;
 * cells of other subdomains give old values. Sources are cells with u = 0 at
 * the start; every other cell starts at +inf (or any upper bound).
 */
typedef struct ndiag_eik ndiag_eik;
typedef struct {
  int sweeps;       /* sweeps run (a multiple of 4) */
  int converged;    /* 1 if the last round's largest change was <= delta */
  double change;    /* largest |u_new - u_old| over the last round's sweeps */
  double seconds;   /* wall time of the call */
  int64_t launches; /* kernels launched on this handle so far */
} ndiag_eik_info;

/*
 * eikonal_create -- copy the slowness f (HOST, nx*ny doubles, x fastest,
 * finite and >= 0) to the device and split the grid into sub[0] x sub[1]
 * nearly equal subdomains (as ndiag_create). A subdomain may have at most 256
 * rows and 25600 columns (one thread per row).
 * Errors: NDIAG_EINVAL (sizes, h <= 0, f, subdomains too large), NDIAG_ENOMEM.
 */
ndiag_status eikonal_create(ndiag_eik** out, const int64_t n[2], double h, const double* f, const int sub[2],
                            void* cuda_stream);
void eikonal_destroy(ndiag_eik* e);

/*
 * eikonal_sweep -- one decomposed sweep at phase t. u_old and u_new are DEVICE
 * vectors of nx*ny doubles and must differ. If change is not NULL the call
 * waits and stores the largest |u_new - u_old|; otherwise it is asynchronous.
 */
ndiag_status eikonal_sweep(ndiag_eik* e, int64_t t, const double* u_old, double* u_new, double* change);

/*
 * eikonal_solve -- sweeps at phases 0, 1, 2, ... in rounds of four (one pass
 * from each start corner per subdomain) until a round's largest change is
 * <= delta, or max_rounds rounds. u (DEVICE or HOST, detected) holds the start
 * values on entry and the result on return. The handle keeps two device
 * vectors for the rounds. Errors: NDIAG_EINVAL, NDIAG_ENOMEM, NDIAG_ENOCONV
 * (max_rounds reached; u holds the last iterate).
 */
ndiag_status eikonal_solve(ndiag_eik* e, double* u, double delta, int max_rounds, ndiag_eik_info* info);

/*
 * ilu0_factor -- ILU(0) (Sec. 5: one symmetric Gauss-Seidel pass on an
 * n-diagonal matrix is ILU(0)). DECOMPOSED: M = (D~ + L_J) D~^-1 (D~ + U_J),
 * L_J / U_J = implicit entries of the forward phase / of its reverse, and
 * d~_i = a_ii - sum_{j in J_i, i not in J_j} a_ij a_ji / d~_j (for the 9-point
 * molecule this is D-ILU: the off-diagonals of A are kept). NATURAL: the same
 * with one lexicographic subdomain for 5/7-point matrices; for 9-point
 * matrices the true ILU(0) of the lexicographic order, whose off-diagonal
 * entries are modified too (IKJ elimination on the 9-point pattern, Saad
 * Alg. 10.4), applied as (D + L') D^-1 (D + U') with D = diag(U). A 5-point
 * matrix stored as a 9-point one with zero corner entries gets its ILU(1)
 * this way: in natural order its level-1 fill is exactly the (x+1, y-1) and
 * (x-1, y+1) positions, and the other corners never fill.
 * DECOMPOSED_FULL: inside every subdomain the true ILU(0) of A's diagonal
 * block in the order that subdomain's forward sweep visits it (its
 * lexicographic order reflected along the axes it sweeps backwards), IKJ on
 * the stencil pattern as above; entries into another subdomain keep A's
 * values, and the apply couples across interfaces as the decomposed sweep
 * does (mutual face pairs solved together). Applied as (D + L') D^-1 (D + U')
 * with the decomposed sweeps of the forward phase and its reverse. With one
 * subdomain it is the natural 9-point factor; a 5-point matrix in 9-point
 * storage gets the decomposed ILU(1); on 5/7-point matrices it equals
 * DECOMPOSED (only the pivots change).
 * Errors: NDIAG_EBREAKDOWN on a zero pivot (reported at the next sync).
 */
ndiag_status ilu0_factor(ndiag* h, int mode);

/* ilu0_apply -- z = M^-1 r: (D~ + L_J) y = r, then (D~ + U_J) z = D~ y.
 * r, z DEVICE vectors (handle precision); z may alias r. ESTATE if not factored. */
ndiag_status ilu0_apply(ndiag* h, const void* r, void* z);

/*
 * ilu0_apply_noalloc -- the same z = M^-1 r as ilu0_apply, for callers that
 * cannot let the library allocate device memory during the call (device
 * memory owned by another allocator or runtime, service loops that must not
 * allocate once running, work replayed from a recorded command stream). The
 * paper has no counterpart: this is an interface variant, not a method step.
 * ilu0_apply allocates its scratch (the intermediate vector y and, for
 * subdomains taller than one slab, the slab hand-off words) on first use; this
 * entry point takes them from one fixed array in device memory instead,
 * NDIAG_NOALLOC_MAX_CELLS cells of fp64 plus 64 Ki hand-off words (about
 * 8.8 MiB), which every GPU that loads the library holds until the process
 * exits. It calls no cudaMalloc, cudaFree or other allocating routine.
 *   r, z   DEVICE vectors (handle precision); z may alias r.
 *   Set-up: the first call on a device looks up the array's device address
 *   with that device current; make that first call before any stream capture.
 *   Later calls look the address up again whenever the handle's stream is not
 *   capturing, so a device reset between calls is picked up.
 *   Sharing: every call uses the same array and leaves its contents behind
 *   (the hand-off words are cleared by each call before use). Calls that
 *   overlap on the GPU (other streams, threads or handles) race on it.
 * Errors: NDIAG_EINVAL if N > NDIAG_NOALLOC_MAX_CELLS, for stencils other than
 * 2D 5-point, or if a subdomain split needs more than 64 Ki hand-off words;
 * NDIAG_ESTATE before ilu0_factor.
 */
#define NDIAG_NOALLOC_MAX_CELLS (1 << 20)
ndiag_status ilu0_apply_noalloc(ndiag* h, const void* r, void* z);

/* Residual r = b - A x in fp64 (A in fp64) and, if norm2 != NULL, ||r||_2
 * copied to the host (synchronises). b, x, r: DEVICE double vectors. */
ndiag_status ndiag_residual(ndiag* h, const double* b, const double* x, double* r, double* norm2);

typedef struct {
  int iterations;        /* Krylov iterations / sweeps / inner iterations in total */
  int outer;             /* refinement steps (1 without refinement) */
  double relres;         /* final TRUE fp64 ||b - A x|| / ||b|| */
  double seconds;        /* wall time of the call */
  int status;            /* same as the return value */
} ndiag_solve_info;

/*
 * krylov_solve -- solve A x = b to ||b - A x||_2 / ||b||_2 <= rtol.
 *   method  NDIAG_PCG, NDIAG_BICGSTAB or NDIAG_STATIONARY (SOR sweeps of the
 *           schedule t = 0, 1, 2, ..., omega[] per direction).
 *   precond NDIAG_PREC_NONE / SSOR / ILU0 / MG (ignored for STATIONARY).
 *           MG: one symmetric multigrid V-cycle with the decomposed SSOR apply
 *           (factor omega[0]) as pre- and post-smoother on every level (the
 *           sweep as a multigrid smoother, Sec. 5). Coarse levels are the
 *           Galerkin products P^T A P over 2 x 2 (x 2) cell aggregates
 *           (piecewise-constant P, so every level stays 5-point / 7-point),
 *           down to a grid of at most 32 (3D: 16) cells per side, where 4 SSOR
 *           steps are taken. 2D 5-point and 3D 7-point fp64 handles and
 *           DECOMPOSED mode only (else NDIAG_EINVAL). The hierarchy is built on the host from the
 *           handle's matrix on the first MG solve, kept on the handle and
 *           freed by ndiag_destroy.
 *   mode    NDIAG_DECOMPOSED or NDIAG_NATURAL ordering of the sweeps.
 *   omega   HOST array of 2^dim relaxation factors (STATIONARY), omega[0] is
 *           the SSOR factor.
 *   b, x    fp64 vectors, DEVICE or HOST pointers (detected); x holds the
 *           initial guess and receives the solution.
 * Stop rule: the recurrence residual meets rtol, then the true fp64 residual is
 * checked; if it is above rtol the method restarts from it. PCG and BiCGSTAB
 * make their stop tests on the device and the host reads the scalars once per
 * chunk of 8 iterations; after the first chunk each chunk is replayed as one
 * captured CUDA graph (not while ndiag_profile is on, and not with the
 * multigrid preconditioner). Iterations the device enqueues after it stopped
 * leave x unchanged. With precision
 * FP32/FP32_D16 the solve is an fp64 iterative refinement around fp32 inner
 * solves; each inner solve aims at the outer tolerance in one go, relative
 * 0.5 rtol ||b|| / ||r|| clamped to [1e-6, 1e-3], at most 60 outer steps.
 * Errors: NDIAG_ENOCONV (maxit), NDIAG_EBREAKDOWN, NDIAG_ESTATE (ILU0 not factored).
 */
ndiag_status krylov_solve(ndiag* h, int method, int precond, int mode, const double* omega,
                          double rtol, int maxit, const double* b, double* x,
                          ndiag_solve_info* info);

/*
 * ndiag_set_history -- record every iteration of the following krylov_solve
 * calls on this handle, so that a solve can be compared with another
 * implementation of the same method iteration by iteration (the residual
 * history before rounding differences grow, Sec. 5 for the preconditioner).
 *   out       HOST array of 4 * capacity doubles, owned by the caller; it must
 *             stay valid until the last solve that records into it returns.
 *             Row k (iteration k + 1) holds, for BiCGSTAB: ||s_k|| / ||b||,
 *             ||r_k|| / ||b||, alpha_k, omega_k (the recurrence vectors of the
 *             two half steps; omega_k = 0 when the half step met the
 *             tolerance); for PCG: ||r_k|| / ||b||, alpha_k, 0, 0. Rows are
 *             written for min(iterations, capacity) iterations, when the solve
 *             returns.
 *   capacity  rows of out; 0 or out = NULL stops recording.
 * Only FP64 handles record (the fp32 inner solves of the refinement do not);
 * the stationary method records nothing. The library allocates a device copy
 * of 32 * capacity bytes, freed by the next call or by ndiag_destroy.
 * Errors: NDIAG_EINVAL (capacity < 0), NDIAG_ENOMEM.
 */
ndiag_status ndiag_set_history(ndiag* h, double* out, int capacity);

/*
 * ndiag_tune_omega -- a relaxation factor per sweep direction for the
 * stationary decomposed SOR iteration. The paper relaxes the sweep directions
 * separately (omega_L, omega_R of Tables 2-5, over- and under-relaxation, with
 * the optimal factors searched in [0, 2]; Theorems 1 and 2 give sufficient
 * conditions for convergence with different factors). This runs a coordinate
 * search over the 2^dim factors (one per start corner, as krylov_solve's
 * omega[]), each trial a full krylov_solve(NDIAG_STATIONARY, DECOMPOSED) from
 * x = 0, minimising the number of sweeps to rtol.
 *   b       fp64 right-hand side, DEVICE or HOST pointer.
 *   rtol, maxit as krylov_solve; a trial that does not converge costs maxit + 1.
 *   budget  the most trial solves to spend (>= 1).
 *   omega   HOST array of 2^dim factors in (0, 2): the start point on entry, the
 *           best factors found on return.
 *   iters   out: sweeps of the returned factors.
 * The library allocates one device vector for the trials and frees it.
 * Errors: NDIAG_EINVAL (arguments), NDIAG_ENOMEM, NDIAG_ENOCONV (no trial
 * converged), or a trial solve's device error.
 */
ndiag_status ndiag_tune_omega(ndiag* h, const double* b, double rtol, int maxit, int budget, double* omega,
                              int* iters);

/*
 * Counters of the library's own kernels on a handle, for measurement.
 *  launches        kernels the library launched since the last ndiag_profile
 *  sweep_launches  sweep kernels among them (one sweep = N cell updates; an
 *                  ILU(0) or SSOR apply is two)
 *  sweep_ms        summed device time of those sweep kernels, from CUDA events
 *                  recorded on the handle's stream around each of them
 *                  (only while profiling is enabled, else 0)
 *  sweep_bytes     algorithmic bytes of those sweeps: every coefficient and
 *                  vector value a sweep must read or write, once per cell
 */
typedef struct {
  int64_t launches;
  int64_t sweep_launches;
  double sweep_ms;
  double sweep_bytes;
} ndiag_counters;

/* Resets the counters; enable != 0 also times every sweep kernel. */
ndiag_status ndiag_profile(ndiag* h, int enable);
/* Synchronises the handle's stream and reports the counters. */
ndiag_status ndiag_read_counters(ndiag* h, ndiag_counters* out);

/*
 * ndiag_set_wavefront -- on != 0 (default): the warp-synchronous wavefront
 * kernels run (lane = row) where they apply: the fp64 decomposed 9-point
 * triangular sweeps (the ILU(0) apply; packed coefficient copy built on first
 * use per coefficient set and phase; subdomains up to 129 rows) and the
 * one-cell part of the 3D 7-point triangular sweeps (a warp per plane;
 * subdomains up to 32 x 32 in y and z). on == 0: the level-by-level kernels.
 * Both compute the same sweep (Secs. 3, 4); their roundings differ.
 */
ndiag_status ndiag_set_wavefront(ndiag* h, int on);

/*
 * Batched solves of many independent 2D 5-point problems (the paper has no
 * counterpart: a GPU serving pattern around its decomposed SSOR). Each problem
 * is a diagonal-major matrix (5 x nx[p]*ny[p], HOST, caller keeps ownership);
 * all vectors of the batch are concatenated in problem order (problem p's
 * cells after those of problems 0..p-1).
 *   ndiag_batch_create   copies the matrices (fp32 sweeps, fp64 matrix for
 *                        residuals); tile[p] = side of the square subdomains of
 *                        problem p (NULL: 64; sides of at most 128); omega =
 *                        SSOR factor; stream NULL = a stream of its own.
 *   ndiag_batch_autotune chooses one tile side for the whole batch from
 *                        {32, 64, 128}: batched SSOR apply time x pilot CG
 *                        iterations (b: DEVICE, concatenated right-hand sides).
 *   ndiag_batch_tiles    reports the tile side of every problem.
 *   ndiag_batch_solve    FP32 SSOR-PCG with FP64 refinement of every problem
 *                        to ||b - A x|| / ||b|| <= rtol (maxit inner
 *                        iterations per refinement step); b, x DEVICE double,
 *                        concatenated; x holds the initial guess; infos[p]
 *                        (HOST, count entries) per problem. Every step of an
 *                        iteration is one launch over all problems; the inner
 *                        iterations of a refinement step are one launch of a
 *                        CUDA graph whose conditional while node runs until
 *                        no problem is active.
 *                        NDIAG_ENOCONV if some problem missed rtol.
 *   ndiag_batch_ssor_apply one application of the batch's preconditioner, the
 *                        decomposed SSOR of Sec. 5 (SPD form, factor omega,
 *                        fp32) of every problem in one launch per pass:
 *                        z = M^-1 r; r, z DEVICE float, concatenated; z must
 *                        not alias r. Synchronises.
 */
typedef struct ndiag_batch ndiag_batch;
ndiag_status ndiag_batch_create(ndiag_batch** out, int count, const int64_t* nx, const int64_t* ny,
                                const double* const* diags, const int* tile, double omega, void* stream);
ndiag_status ndiag_batch_autotune(ndiag_batch* b, const double* rhs);
ndiag_status ndiag_batch_tiles(const ndiag_batch* b, int* tile);
ndiag_status ndiag_batch_solve(ndiag_batch* b, double rtol, int maxit, const double* rhs, double* x,
                               ndiag_solve_info* infos);
ndiag_status ndiag_batch_ssor_apply(ndiag_batch* b, const float* r, float* z);
int64_t ndiag_batch_cells(const ndiag_batch* b);
int64_t ndiag_batch_launches(const ndiag_batch* b);
void ndiag_batch_destroy(ndiag_batch* b);

/*
 * Solve server with continuous batching (no counterpart in the paper).
 *   ndiag_server_create  slots = concurrent solves (worker threads, each with
 *                        its own CUDA stream, 1..64); mem_budget = device
 *                        bytes the running solves may hold (0: 80 % of the
 *                        free memory now).
 *   serve_submit         copies the request (HOST diags s x N and b) and
 *                        queues it; *ticket identifies it. A queued request is
 *                        admitted when a slot is free and its estimated memory
 *                        fits the remaining budget (first fitting request in
 *                        arrival order; one larger than the whole budget runs
 *                        alone). Always decomposed ordering with sub[];
 *                        ILU0 requests are factored first, with
 *                        DECOMPOSED_FULL (on 9-point matrices the full ILU(0)
 *                        of every subdomain block; 5/7-point: DECOMPOSED).
 *   serve_poll           NDIAG_EBUSY while the request is queued or running;
 *                        then fills *out, copies x (HOST, N doubles) if x is
 *                        not NULL, and forgets the ticket.
 *   ndiag_server_wait    blocks until the request is done or timeout_s passed
 *                        (NDIAG_EBUSY).
 *   ndiag_server_destroy finishes the queued requests, then stops.
 */
typedef struct ndiag_server ndiag_server;
typedef struct {
  int dim, stencil;
  int64_t n[3];
  int sub[3];
  const double* diags; /* HOST, stencil x N, diagonal-major */
  const double* b;     /* HOST, N */
  int method, precond, precision;
  double rtol;
  int maxit;
  double omega;        /* SSOR factor (<= 0: 1) */
} ndiag_request;
typedef struct {
  int status;
  ndiag_solve_info info;
  double queue_s, run_s, latency_s; /* submit -> start, start -> end, submit -> end */
  int64_t cells;
} ndiag_result;
typedef struct {
  int queued, running, max_running;
  int64_t solved, budget_bytes, in_use_bytes;
} ndiag_server_stats_t;
ndiag_status ndiag_server_create(ndiag_server** out, int slots, size_t mem_budget);
ndiag_status serve_submit(ndiag_server* s, const ndiag_request* req, uint64_t* ticket);
ndiag_status serve_poll(ndiag_server* s, uint64_t ticket, ndiag_result* out, double* x);
ndiag_status ndiag_server_wait(ndiag_server* s, uint64_t ticket, double timeout_s);
ndiag_status ndiag_server_stats(ndiag_server* s, ndiag_server_stats_t* out);
void ndiag_server_destroy(ndiag_server* s);

#ifdef __cplusplus
}
#endif

#endif /* NDIAG_H */
