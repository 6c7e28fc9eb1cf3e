"""CPU oracle of the decomposed sequential sweep (test infrastructure).

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
legs may import this package. It wraps oracle/oracle.cpp (plain single-threaded
fp64 C++, see that file's header for the paper passage behind every function)
through ctypes. It shares no code with the CUDA library.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

NATURAL, DECOMPOSED = 0, 1
# ilu0_factor only: the decomposed ordering with the full ILU(0) of the stencil
# pattern inside every subdomain (modified off-diagonals; 9-point molecules)
DECOMPOSED_FULL = 3
PREC_NONE, PREC_SSOR, PREC_ILU0 = 0, 1, 2
PCG, BICGSTAB, STATIONARY = 0, 1, 2


def build(force: bool = False, extra_flags: tuple[str, ...] = (), out: str | None = None) -> str:
    """Compile oracle.cpp into a shared library (plain g++, fp64, no FMA
    contraction, no fast-math)."""
    out = out or _LIB_PATH
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    cmd = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           *extra_flags, "-o", out, _SRC]
    subprocess.run(cmd, check=True)
    return out


def _load(path: str):
    lib = ctypes.CDLL(path)
    P, I, L, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    lib.orc_create.restype = P
    lib.orc_create.argtypes = [I, P, I, P, P]
    lib.orc_destroy.argtypes = [P]
    lib.orc_ncells.restype = L
    lib.orc_ncells.argtypes = [P]
    lib.orc_base_corner.restype = I
    lib.orc_base_corner.argtypes = [I, L]
    lib.orc_matvec.argtypes = [P, P, P]
    lib.orc_plan_info.argtypes = [P, I, L, P, P, P, P]
    lib.orc_sor_sweep.argtypes = [P, I, L, P, P, P, P]
    lib.orc_ilu0_factor.argtypes = [P, I]
    lib.orc_ilu0_export.argtypes = [P, P]
    lib.orc_ilu0_apply.argtypes = [P, P, P]
    lib.orc_ssor_apply.argtypes = [P, I, D, P, P]
    lib.orc_fwd_phase.restype = I
    lib.orc_fwd_phase.argtypes = [I]
    lib.orc_solve.argtypes = [P, I, I, I, P, D, I, P, P, P]
    lib.orc_history.argtypes = [P, P, L]
    lib.orc_history.restype = L
    lib.orc_eik_create.restype = P
    lib.orc_eik_create.argtypes = [P, D, P, P]
    lib.orc_eik_destroy.argtypes = [P]
    lib.orc_eik_sweep.argtypes = [P, L, P, P, P]
    lib.orc_eik_solve.argtypes = [P, P, D, I, P]
    return lib


def lib(path: str | None = None):
    global _lib
    if path is not None:
        return _load(path)
    if _lib is None:
        build()
        _lib = _load(_LIB_PATH)
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _omega8(omega) -> np.ndarray:
    """Relaxation factor per sweep direction (start corner 0..2^d-1); a scalar
    applies to every direction."""
    v = np.atleast_1d(np.asarray(omega, dtype=np.float64)).ravel()
    om = np.zeros(8)
    if len(v) == 1:
        om[:] = v[0]
    else:
        om[: len(v)] = v
    return om


class Problem:
    """One structured n-diagonal system A u = b on a Cartesian grid split into
    sub[0] x sub[1] x sub[2] subdomains."""

    def __init__(self, dim, n, stencil, diags, sub=(1, 1, 1), library=None):
        self.lib = library or lib()
        self.dim = int(dim)
        self.n = tuple(int(v) for v in (list(n) + [1, 1, 1])[:3])
        self.stencil = int(stencil)
        self.N = int(np.prod(self.n[: self.dim]))
        self.diags = _f64(diags).reshape(self.stencil, self.N)
        n64 = np.array(self.n, dtype=np.int64)
        sub32 = np.array((list(sub) + [1, 1, 1])[:3], dtype=np.int32)
        self.sub = tuple(int(v) for v in sub32)
        self.h = self.lib.orc_create(self.dim, _ptr(n64), self.stencil, _ptr(self.diags), _ptr(sub32))
        if not self.h:
            raise ValueError("oracle: bad grid/stencil/subdomains")

    def __del__(self):
        if getattr(self, "h", None):
            self.lib.orc_destroy(self.h)
            self.h = None

    def matvec(self, x):
        x = _f64(x)
        y = np.empty(self.N)
        self.lib.orc_matvec(self.h, _ptr(x), _ptr(y))
        return y

    def plan_info(self, mode, t):
        jm = np.empty(self.N, dtype=np.uint16)
        cr = np.empty(self.N, dtype=np.uint8)
        nb = ctypes.c_int64()
        mb = ctypes.c_int64()
        self.lib.orc_plan_info(self.h, mode, t, _ptr(jm), _ptr(cr), ctypes.byref(nb), ctypes.byref(mb))
        return jm, cr, nb.value, mb.value

    def sor_sweep(self, mode, t, omega, b, x_old):
        om = _omega8(omega)
        b = _f64(b)
        x_old = _f64(x_old)
        x_new = np.empty(self.N)
        rc = self.lib.orc_sor_sweep(self.h, mode, t, _ptr(om), _ptr(b), _ptr(x_old), _ptr(x_new))
        if rc:
            raise RuntimeError("oracle sweep failed")
        return x_new

    def ilu0_factor(self, mode):
        if self.lib.orc_ilu0_factor(self.h, mode):
            raise RuntimeError("oracle ILU(0) failed")
        self.ilu_mode = mode

    def ilu0_export(self):
        out = np.empty(self.N if self.ilu_mode == DECOMPOSED else self.stencil * self.N)
        self.lib.orc_ilu0_export(self.h, _ptr(out))
        return out if self.ilu_mode == DECOMPOSED else out.reshape(self.stencil, self.N)

    def ilu0_apply(self, r):
        r = _f64(r)
        z = np.empty(self.N)
        if self.lib.orc_ilu0_apply(self.h, _ptr(r), _ptr(z)):
            raise RuntimeError("oracle ILU(0) apply failed")
        return z

    def ssor_apply(self, mode, omega, r):
        r = _f64(r)
        z = np.empty(self.N)
        if self.lib.orc_ssor_apply(self.h, mode, float(omega), _ptr(r), _ptr(z)):
            raise RuntimeError("oracle SSOR apply failed")
        return z

    def fwd_phase(self):
        return self.lib.orc_fwd_phase(self.dim)

    def solve(self, method, precond, mode, omega, rtol, maxit, b, x0=None):
        om = _omega8(omega)
        b = _f64(b)
        x = np.zeros(self.N) if x0 is None else _f64(x0).copy()
        info = np.zeros(3)
        rc = self.lib.orc_solve(self.h, method, precond, mode, _ptr(om), float(rtol), int(maxit),
                                _ptr(b), _ptr(x), _ptr(info))
        if rc:
            raise RuntimeError(f"oracle solve failed ({rc})")
        out = dict(iters=int(info[0]), relres=float(info[1]), status=int(info[2]))
        # per-iteration record (BiCGSTAB: ||s||/||b||, ||r||/||b||, alpha, omega;
        # PCG: ||r||/||b||, alpha, 0, 0)
        rows = self.lib.orc_history(self.h, None, 0)
        hist = np.zeros((rows, 4))
        if rows:
            self.lib.orc_history(self.h, _ptr(hist), rows)
        out["history"] = hist
        return x, out


class Eikonal:
    """Fast sweeping for |grad u| = f on an nx x ny grid of spacing h, split
    into sub[0] x sub[1] subdomains (decomposed Gauss-Seidel passes)."""

    def __init__(self, n, h, f, sub=(1, 1), library=None):
        self.lib = library or lib()
        self.n = (int(n[0]), int(n[1]))
        self.N = self.n[0] * self.n[1]
        self.f = _f64(f).reshape(self.N)
        n64 = np.array(self.n, dtype=np.int64)
        sub32 = np.array(list(sub)[:2], dtype=np.int32)
        self.h = self.lib.orc_eik_create(_ptr(n64), float(h), _ptr(self.f), _ptr(sub32))
        if not self.h:
            raise ValueError("oracle: bad eikonal grid/subdomains")

    def __del__(self):
        if getattr(self, "h", None):
            self.lib.orc_eik_destroy(self.h)
            self.h = None

    def sweep(self, t, u_old):
        u_old = _f64(u_old)
        u_new = np.empty(self.N)
        ch = ctypes.c_double()
        self.lib.orc_eik_sweep(self.h, int(t), _ptr(u_old), _ptr(u_new), ctypes.byref(ch))
        return u_new, ch.value

    def solve(self, u0, delta=0.0, max_rounds=1000):
        u = _f64(u0).copy()
        info = np.zeros(3)
        self.lib.orc_eik_solve(self.h, _ptr(u), float(delta), int(max_rounds), _ptr(info))
        return u, dict(sweeps=int(info[0]), change=float(info[1]), converged=bool(info[2]))


def eikonal_init(n_cells: int, sources) -> np.ndarray:
    """u0: 0 at the source cells, +inf elsewhere."""
    u = np.full(n_cells, np.inf)
    u[np.asarray(sources, dtype=np.int64)] = 0.0
    return u


def base_corner(dim: int, t: int) -> int:
    return lib().orc_base_corner(dim, t)
