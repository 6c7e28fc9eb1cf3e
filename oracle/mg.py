"""Oracle of the multigrid V-cycle preconditioner (test infrastructure).

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
legs may import this module. It shares no code with the CUDA library.

The paper (Sec. 5, opening paragraph) names the use of SOR as a smoother in
multigrid methods, a few sweeps per smoothing step, as one of the main uses of
the sweep; it gives no cycle. The cycle here is the textbook symmetric V(1,1)
cycle used as a PCG preconditioner, written in the plainest form:

  hierarchy  level 0 is the given 2D 5-point problem; level k+1 is the Galerkin
             product A_{k+1} = P_k^T A_k P_k, where P_k is the piecewise-constant
             prolongation over 2 x 2 aggregates of cells (cell (x, y) belongs to
             aggregate (x // 2, y // 2); the last aggregate of an odd side is one
             cell wide). A_{k+1} keeps the 5-point pattern. Coarsening stops once
             both sides are at most 32 cells, or after 10 levels.
  partition  level 0 keeps the caller's subdomains; a coarse level of
             nx x ny cells is split into min(16, max(1, nx // 16)) x
             min(16, max(1, ny // 16)) subdomains.
  smoother   S_k = the decomposed SSOR apply of level k (Sec. 2: SSOR = a sweep
             and its reverse, in the SPD form), factor omega.
  cycle      B_k r:  z  = S_k r
                     z += ALPHA P_k B_{k+1} P_k^T (r - A_k z)
                     z += S_k (r - A_k z)
             and on the coarsest level KC = 4 steps of SSOR-Richardson,
             z = S r, then z += S (r - A z) three times. ALPHA = 1.8 is the
             usual over-correction of a piecewise-constant (unsmoothed
             aggregation) coarse correction, whose Galerkin operator is about
             twice too stiff for smooth error (Braess 1995; Notay and
             Vassilevski 2008); it keeps B symmetric.
  smoother factor  omega must stay below 1 when subdomains meet at interior
             vertices: the coupled start-corner blocks of the decomposed sweep
             give S A an eigenvalue of exactly 2 at omega = 1 (more beyond), so
             the smoother stops contracting in the A-norm there.
  Krylov     PCG with the stop rule of the C++ oracle: the recurrence residual
             meets rtol, then the true residual is checked and the method
             restarts from it if it is above rtol.

The sparse products are scipy's (a library primitive standing for P^T A P);
the SSOR apply and the matrix-vector product are the C++ oracle's.
The 3D 7-point cycle (Hierarchy3) is the same with 2 x 2 x 2 aggregates,
coarsening while a side exceeds 16 cells and coarse parts min(8, max(1, n // 16)).

Pins: tests/test_oracle_mg.py (dense P^T A P, the closed form of the Poisson
coarse stencil, the dense error-propagation form of the two-level cycle, the
closed form of SSOR-Richardson, symmetry and definiteness; the 3D cycle's
Galerkin product, coarse stencil, two-level form and smoother bound).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp

import oracle

KC = 4          # SSOR-Richardson steps on the coarsest level
ALPHA = 1.8     # over-correction of the coarse-grid correction
NMIN = 32       # coarsen while a side exceeds this
LMAX = 10       # levels at most

def coarse_parts(n: int) -> int:
    """Subdomains along an axis of n cells on a coarse level."""
    return min(16, max(1, n // 16))


def prolongation(nx: int, ny: int) -> sp.csr_matrix:
    """P (nx*ny x nxc*nyc): P[i, I] = 1 when fine cell i lies in aggregate I."""
    nxc, nyc = (nx + 1) // 2, (ny + 1) // 2
    i = np.arange(nx * ny)
    x, y = i % nx, i // nx
    I = (y // 2) * nxc + x // 2
    return sp.csr_matrix((np.ones(nx * ny), (i, I)), shape=(nx * ny, nxc * nyc))


def to_sparse(nx: int, ny: int, diags: np.ndarray) -> sp.csr_matrix:
    """The 5-point matrix of diagonal-major entries C W E S N (x fastest)."""
    N = nx * ny
    i = np.arange(N)
    x, y = i % nx, i // nx
    rows, cols, vals = [i], [i], [diags[0]]
    for k, (dx, dy) in enumerate(((-1, 0), (1, 0), (0, -1), (0, 1)), start=1):
        ok = (x + dx >= 0) & (x + dx < nx) & (y + dy >= 0) & (y + dy < ny)
        rows.append(i[ok])
        cols.append(i[ok] + dx + dy * nx)
        vals.append(diags[k][ok])
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(N, N))


def from_sparse(nx: int, ny: int, A: sp.spmatrix) -> np.ndarray:
    """Diagonal-major 5-point entries of A; raises if A has entries elsewhere."""
    A = sp.coo_matrix(A)
    N = nx * ny
    r, c = A.row.astype(np.int64), A.col.astype(np.int64)
    dx, dy = c % nx - r % nx, c // nx - r // nx
    k = np.full(r.shape, -1)
    for kk, (ox, oy) in enumerate(((0, 0), (-1, 0), (1, 0), (0, -1), (0, 1))):
        k[(dx == ox) & (dy == oy)] = kk
    if np.any((k < 0) & (A.data != 0.0)):
        raise ValueError("coarse operator left the 5-point pattern")
    d = np.zeros((5, N))
    keep = k >= 0
    np.add.at(d, (k[keep], r[keep]), A.data[keep])
    return d


def galerkin(nx: int, ny: int, diags: np.ndarray) -> np.ndarray:
    """A_c = P^T A P as diagonal-major 5-point entries of the coarse grid."""
    P = prolongation(nx, ny)
    C = (P.T @ to_sparse(nx, ny, diags) @ P).tocoo()
    return from_sparse((nx + 1) // 2, (ny + 1) // 2, C)


class Hierarchy:
    """Levels (nx, ny, oracle.Problem) from the fine grid down."""

    def __init__(self, nx, ny, diags, sub, omega, library=None):
        self.omega = float(omega)
        self.levels = [(nx, ny, oracle.Problem(2, (nx, ny), 5, diags, (sub[0], sub[1]), library=library))]
        d = np.asarray(diags, dtype=np.float64).reshape(5, nx * ny)
        while (nx > NMIN or ny > NMIN) and len(self.levels) < LMAX:
            d = galerkin(nx, ny, d)
            nx, ny = (nx + 1) // 2, (ny + 1) // 2
            sub_c = (coarse_parts(nx), coarse_parts(ny))
            self.levels.append((nx, ny, oracle.Problem(2, (nx, ny), 5, d, sub_c, library=library)))

    def smooth(self, k, r):
        return self.levels[k][2].ssor_apply(oracle.DECOMPOSED, self.omega, r)

    def vcycle(self, r, k=0):
        nx, ny, pb = self.levels[k]
        z = self.smooth(k, r)
        if k + 1 == len(self.levels):
            for _ in range(KC - 1):
                z = z + self.smooth(k, r - pb.matvec(z))
            return z
        P = self.prolong(k)
        z = z + ALPHA * (P @ self.vcycle(P.T @ (r - pb.matvec(z)), k + 1))
        return z + self.smooth(k, r - pb.matvec(z))

    def prolong(self, k):
        nx, ny, _ = self.levels[k]
        return prolongation(nx, ny)


def pcg(H: Hierarchy, b, rtol, maxit, x0=None):
    """PCG preconditioned by one V-cycle; returns x and the oracle's info dict."""
    pb = H.levels[0][2]
    b = np.asarray(b, dtype=np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    bnorm = math.sqrt(b @ b)
    if bnorm == 0.0:
        return np.zeros_like(b), dict(iters=0, relres=0.0, status=0)
    it = 0
    while True:
        r = b - pb.matvec(x)
        rel = math.sqrt(r @ r) / bnorm
        if rel <= rtol:
            return x, dict(iters=it, relres=rel, status=0)
        z = H.vcycle(r)
        p = z.copy()
        rz = r @ z
        recheck = False
        while it < maxit:
            Ap = pb.matvec(p)
            pAp = p @ Ap
            if pAp == 0.0 or rz == 0.0:
                rr = b - pb.matvec(x)
                return x, dict(iters=it, relres=math.sqrt(rr @ rr) / bnorm, status=2)
            alpha = rz / pAp
            x = x + alpha * p
            r = r - alpha * Ap
            it += 1
            if math.sqrt(r @ r) / bnorm <= rtol:
                recheck = True
                break
            z = H.vcycle(r)
            rz2 = r @ z
            p = z + (rz2 / rz) * p
            rz = rz2
        rr = b - pb.matvec(x)
        tr = math.sqrt(rr @ rr) / bnorm
        if not recheck:
            return x, dict(iters=it, relres=tr, status=1)
        if tr <= rtol:
            return x, dict(iters=it, relres=tr, status=0)


# --- 3D 7-point ------------------------------------------------------------
# The same cycle on 7-point matrices (entries C W E S N B F, x fastest):
# 2 x 2 x 2 aggregates (one cell wide at an odd side's end), coarsening while a
# side exceeds NMIN3, coarse levels split into coarse_parts3(n) parts per axis.

NMIN3 = 16


def coarse_parts3(n: int) -> int:
    """Subdomains along an axis of n cells on a coarse 3D level."""
    return min(8, max(1, n // 16))


_OFF7 = ((0, 0, 0), (-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1))


def prolongation3(n) -> sp.csr_matrix:
    """P (N x Nc): P[i, I] = 1 when fine cell i lies in aggregate I."""
    nx, ny, nz = n
    nxc, nyc, nzc = (nx + 1) // 2, (ny + 1) // 2, (nz + 1) // 2
    i = np.arange(nx * ny * nz)
    x, y, z = i % nx, (i // nx) % ny, i // (nx * ny)
    I = ((z // 2) * nyc + y // 2) * nxc + x // 2
    return sp.csr_matrix((np.ones(i.size), (i, I)), shape=(i.size, nxc * nyc * nzc))


def to_sparse3(n, diags: np.ndarray) -> sp.csr_matrix:
    """The 7-point matrix of diagonal-major entries."""
    nx, ny, nz = n
    N = nx * ny * nz
    i = np.arange(N)
    x, y, z = i % nx, (i // nx) % ny, i // (nx * ny)
    rows, cols, vals = [], [], []
    for k, (dx, dy, dz) in enumerate(_OFF7):
        ok = (x + dx >= 0) & (x + dx < nx) & (y + dy >= 0) & (y + dy < ny) & (z + dz >= 0) & (z + dz < nz)
        rows.append(i[ok])
        cols.append(i[ok] + dx + nx * (dy + ny * dz))
        vals.append(diags[k][ok])
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(N, N))


def from_sparse3(n, A: sp.spmatrix) -> np.ndarray:
    """Diagonal-major 7-point entries of A; raises if A has entries elsewhere."""
    nx, ny, nz = n
    A = sp.coo_matrix(A)
    r, c = A.row.astype(np.int64), A.col.astype(np.int64)
    dx = c % nx - r % nx
    dy = (c // nx) % ny - (r // nx) % ny
    dz = c // (nx * ny) - r // (nx * ny)
    k = np.full(r.shape, -1)
    for kk, (ox, oy, oz) in enumerate(_OFF7):
        k[(dx == ox) & (dy == oy) & (dz == oz)] = kk
    if np.any((k < 0) & (A.data != 0.0)):
        raise ValueError("coarse operator left the 7-point pattern")
    d = np.zeros((7, nx * ny * nz))
    keep = k >= 0
    np.add.at(d, (k[keep], r[keep]), A.data[keep])
    return d


def galerkin3(n, diags: np.ndarray) -> np.ndarray:
    """A_c = P^T A P as diagonal-major 7-point entries of the coarse grid."""
    P = prolongation3(n)
    C = (P.T @ to_sparse3(n, diags) @ P).tocoo()
    return from_sparse3(tuple((v + 1) // 2 for v in n), C)


class Hierarchy3(Hierarchy):
    """Levels (n, None, oracle.Problem) of a 3D 7-point problem."""

    def __init__(self, n, diags, sub, omega, library=None):
        self.omega = float(omega)
        n = tuple(int(v) for v in n)
        self.levels = [(n, None, oracle.Problem(3, n, 7, diags, tuple(sub), library=library))]
        d = np.asarray(diags, dtype=np.float64).reshape(7, int(np.prod(n)))
        while max(n) > NMIN3 and len(self.levels) < LMAX:
            d = galerkin3(n, d)
            n = tuple((v + 1) // 2 for v in n)
            sub_c = tuple(coarse_parts3(v) for v in n)
            self.levels.append((n, None, oracle.Problem(3, n, 7, d, sub_c, library=library)))

    def prolong(self, k):
        return prolongation3(self.levels[k][0])
