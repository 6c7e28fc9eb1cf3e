"""Python binding of libndiag.so (include/ndiag.h): argument marshalling only.

Every step of a sweep, factorisation or solve runs in the CUDA library; this
module converts torch tensors / numpy arrays to pointers and status codes to
exceptions. Device memory that the library allocates comes from torch's
caching allocator through the C allocator hook. There is no CPU fallback: if
the library is missing, importing the binding's entry points fails loudly.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libndiag.so")

OK, EINVAL, ENOMEM, ENOCONV, EBREAKDOWN, EDEVICE, ETIMEOUT, EBUSY, ESTATE = range(9)
STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "ENOCONV", "EBREAKDOWN", "EDEVICE", "ETIMEOUT", "EBUSY", "ESTATE"]
FP64, FP32, FP32_D16 = 0, 1, 2
PRECISION = {"fp64": FP64, "fp32": FP32, "fp32_d16": FP32_D16}
NATURAL, DECOMPOSED = 0, 1
# ilu0_factor only: full ILU(0) of every subdomain block (9-point: modified off-diagonals)
DECOMPOSED_FULL = 3
PCG, BICGSTAB, STATIONARY = 0, 1, 2
PREC_NONE, PREC_SSOR, PREC_ILU0, PREC_MG = 0, 1, 2, 3

# every symbol include/ndiag.h declares
EXPORTED = ["ndiag_set_allocator", "ndiag_last_error", "ndiag_create", "ndiag_destroy", "ndiag_cells",
            "ndiag_precision", "sor_sweep", "ssor_apply", "mg_apply", "ndiag_mg_levels", "ndiag_selftest_wait", "ilu0_factor", "ilu0_apply", "ndiag_residual",
            "krylov_solve", "ndiag_set_history", "ndiag_tune_omega", "ndiag_profile", "ndiag_read_counters", "ilu0_apply_noalloc",
            "ndiag_set_wavefront",
            "ndiag_batch_create", "ndiag_batch_autotune", "ndiag_batch_tiles", "ndiag_batch_solve",
            "ndiag_batch_ssor_apply",
            "ndiag_batch_cells", "ndiag_batch_launches", "ndiag_batch_destroy",
            "ndiag_server_create", "serve_submit", "serve_poll", "ndiag_server_wait", "ndiag_server_stats",
            "ndiag_server_destroy", "eikonal_create", "eikonal_destroy", "eikonal_sweep", "eikonal_solve"]
NOALLOC_MAX_CELLS = 1 << 20


class NdiagError(RuntimeError):
    def __init__(self, status, msg=""):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"ndiag {name}: {msg}")


class SolveInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("outer", ctypes.c_int), ("relres", ctypes.c_double),
                ("seconds", ctypes.c_double), ("status", ctypes.c_int)]


class Request(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("stencil", ctypes.c_int), ("n", ctypes.c_int64 * 3),
                ("sub", ctypes.c_int * 3), ("diags", ctypes.c_void_p), ("b", ctypes.c_void_p),
                ("method", ctypes.c_int), ("precond", ctypes.c_int), ("precision", ctypes.c_int),
                ("rtol", ctypes.c_double), ("maxit", ctypes.c_int), ("omega", ctypes.c_double)]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("info", SolveInfo), ("queue_s", ctypes.c_double),
                ("run_s", ctypes.c_double), ("latency_s", ctypes.c_double), ("cells", ctypes.c_int64)]


class ServerStats(ctypes.Structure):
    _fields_ = [("queued", ctypes.c_int), ("running", ctypes.c_int), ("max_running", ctypes.c_int),
                ("solved", ctypes.c_int64), ("budget_bytes", ctypes.c_int64), ("in_use_bytes", ctypes.c_int64)]


class EikInfo(ctypes.Structure):
    _fields_ = [("sweeps", ctypes.c_int), ("converged", ctypes.c_int), ("change", ctypes.c_double),
                ("seconds", ctypes.c_double), ("launches", ctypes.c_int64)]


class Counters(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("sweep_launches", ctypes.c_int64), ("sweep_ms", ctypes.c_double),
                ("sweep_bytes", ctypes.c_double)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)

_lib = None
_hooks = None


def load(path: str = LIB_PATH):
    """Load libndiag.so (raises if it has not been built)."""
    global _lib
    if _lib is not None and path == LIB_PATH:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with __graft_entry__.build()")
    L = ctypes.CDLL(path)
    P, I, L64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    L.ndiag_set_allocator.argtypes = [ALLOC_FN, FREE_FN, P]
    L.ndiag_last_error.restype = ctypes.c_char_p
    L.ndiag_create.argtypes = [ctypes.POINTER(P), I, P, I, P, P, I, P]
    L.ndiag_destroy.argtypes = [P]
    L.ndiag_destroy.restype = None
    L.ndiag_cells.argtypes = [P]
    L.ndiag_cells.restype = L64
    L.ndiag_precision.argtypes = [P]
    L.sor_sweep.argtypes = [P, I, P, L64, P, P, P]
    L.ssor_apply.argtypes = [P, I, D, P, P]
    L.mg_apply.argtypes = [P, D, P, P]
    L.ndiag_mg_levels.argtypes = [P]
    L.ndiag_selftest_wait.argtypes = [P]
    L.ilu0_factor.argtypes = [P, I]
    L.ilu0_apply.argtypes = [P, P, P]
    L.ilu0_apply_noalloc.argtypes = [P, P, P]
    L.ndiag_residual.argtypes = [P, P, P, P, ctypes.POINTER(D)]
    L.krylov_solve.argtypes = [P, I, I, I, P, D, I, P, P, ctypes.POINTER(SolveInfo)]
    L.ndiag_set_history.argtypes = [P, P, I]
    L.ndiag_tune_omega.argtypes = [P, P, D, I, I, P, ctypes.POINTER(I)]
    L.ndiag_profile.argtypes = [P, I]
    L.ndiag_set_wavefront.argtypes = [P, I]
    L.ndiag_read_counters.argtypes = [P, ctypes.POINTER(Counters)]
    L.ndiag_batch_create.argtypes = [ctypes.POINTER(P), I, P, P, P, P, D, P]
    L.ndiag_batch_autotune.argtypes = [P, P]
    L.ndiag_batch_tiles.argtypes = [P, P]
    L.ndiag_batch_solve.argtypes = [P, D, I, P, P, P]
    L.ndiag_batch_ssor_apply.argtypes = [P, P, P]
    L.ndiag_batch_cells.argtypes = [P]
    L.ndiag_batch_cells.restype = L64
    L.ndiag_batch_launches.argtypes = [P]
    L.ndiag_batch_launches.restype = L64
    L.ndiag_batch_destroy.argtypes = [P]
    L.ndiag_batch_destroy.restype = None
    L.ndiag_server_create.argtypes = [ctypes.POINTER(P), I, ctypes.c_size_t]
    L.serve_submit.argtypes = [P, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)]
    L.serve_poll.argtypes = [P, ctypes.c_uint64, ctypes.POINTER(Result), P]
    L.ndiag_server_wait.argtypes = [P, ctypes.c_uint64, D]
    L.ndiag_server_stats.argtypes = [P, ctypes.POINTER(ServerStats)]
    L.ndiag_server_destroy.argtypes = [P]
    L.ndiag_server_destroy.restype = None
    L.eikonal_create.argtypes = [ctypes.POINTER(P), P, D, P, P, P]
    L.eikonal_destroy.argtypes = [P]
    L.eikonal_destroy.restype = None
    L.eikonal_sweep.argtypes = [P, L64, P, P, P]
    L.eikonal_solve.argtypes = [P, P, D, I, ctypes.POINTER(EikInfo)]
    if path == LIB_PATH:
        _lib = L
    return L


def _install_torch_allocator(L):
    """Route the library's device allocations through torch's caching allocator."""
    global _hooks
    if _hooks is not None:
        return
    import torch

    def alloc(nbytes, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
        except Exception:  # out of memory: the library reports NDIAG_ENOMEM
            return None

    def free(ptr, nbytes, stream, ctx):
        torch.cuda.caching_allocator_delete(int(ptr))

    _hooks = (ALLOC_FN(alloc), FREE_FN(free))
    L.ndiag_set_allocator(_hooks[0], _hooks[1], None)


def _check(L, status):
    if status != OK:
        raise NdiagError(status, L.ndiag_last_error().decode(errors="replace"))


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    return a.ctypes.data_as(ctypes.c_void_p)


def _omega(omega, dim):
    v = np.atleast_1d(np.asarray(omega, dtype=np.float64)).ravel()
    out = np.full(8, v[0]) if len(v) == 1 else np.zeros(8)
    if len(v) > 1:
        out[: len(v)] = v
    return out


class NDiag:
    """A structured n-diagonal system resident on the current CUDA device."""

    def __init__(self, dim, n, stencil, diags, sub=(1, 1, 1), precision="fp64", stream=None):
        import torch
        self.L = load()
        _install_torch_allocator(self.L)
        self.dim = int(dim)
        self.n = tuple(int(v) for v in (list(n) + [1, 1, 1])[:3])
        self.stencil = int(stencil)
        self.N = int(np.prod(self.n[: self.dim]))
        self.precision = PRECISION[precision] if isinstance(precision, str) else int(precision)
        self.dtype = torch.float64 if self.precision == FP64 else torch.float32
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        d = np.ascontiguousarray(diags, dtype=np.float64).reshape(self.stencil, self.N)
        n64 = np.array(self.n, dtype=np.int64)
        sub32 = np.array((list(sub) + [1, 1, 1])[:3], dtype=np.int32)
        self.sub = tuple(int(v) for v in sub32)
        h = ctypes.c_void_p()
        _check(self.L, self.L.ndiag_create(ctypes.byref(h), self.dim, _ptr(n64), self.stencil, _ptr(d),
                                           _ptr(sub32), self.precision, ctypes.c_void_p(self.stream.cuda_stream)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.L.ndiag_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def empty(self, dtype=None):
        import torch
        return torch.empty(self.N, dtype=dtype or self.dtype, device="cuda")

    def sor_sweep(self, omega, t, b, x_old, x_new, mode=DECOMPOSED):
        _check(self.L, self.L.sor_sweep(self.h, mode, _ptr(_omega(omega, self.dim)), int(t), _ptr(b),
                                        _ptr(x_old), _ptr(x_new)))

    def ssor_apply(self, omega, r, z, mode=DECOMPOSED):
        _check(self.L, self.L.ssor_apply(self.h, mode, float(omega), _ptr(r), _ptr(z)))

    def mg_apply(self, omega, r, z):
        """One multigrid V-cycle z = B r (fp64 device tensors)."""
        _check(self.L, self.L.mg_apply(self.h, float(omega), _ptr(r), _ptr(z)))

    def mg_levels(self):
        return int(self.L.ndiag_mg_levels(self.h))

    def selftest_wait(self):
        """Runs the bounded-wait failure path; returns the status name (ETIMEOUT expected)."""
        return STATUS_NAMES[self.L.ndiag_selftest_wait(self.h)]

    def ilu0_factor(self, mode=DECOMPOSED):
        _check(self.L, self.L.ilu0_factor(self.h, mode))

    def ilu0_apply(self, r, z):
        _check(self.L, self.L.ilu0_apply(self.h, _ptr(r), _ptr(z)))

    def ilu0_apply_noalloc(self, r, z):
        """ilu0_apply without device allocation (fixed scratch inside the library)."""
        _check(self.L, self.L.ilu0_apply_noalloc(self.h, _ptr(r), _ptr(z)))

    def residual(self, b, x, r):
        nrm = ctypes.c_double()
        _check(self.L, self.L.ndiag_residual(self.h, _ptr(b), _ptr(x), _ptr(r), ctypes.byref(nrm)))
        return nrm.value

    def set_wavefront(self, on=True):
        """Wavefront kernels (9-point fp64 triangular sweeps, 3D one-cell walks) or the level kernels."""
        _check(self.L, self.L.ndiag_set_wavefront(self.h, 1 if on else 0))

    def profile(self, enable=True):
        """Reset the launch counters; with enable, time every sweep kernel."""
        _check(self.L, self.L.ndiag_profile(self.h, 1 if enable else 0))

    def counters(self):
        c = Counters()
        _check(self.L, self.L.ndiag_read_counters(self.h, ctypes.byref(c)))
        return dict(launches=c.launches, sweep_launches=c.sweep_launches, sweep_ms=c.sweep_ms,
                    sweep_bytes=c.sweep_bytes)

    def solve(self, method, precond, b, x, rtol=1e-8, maxit=10000, omega=1.0, mode=DECOMPOSED,
              raise_on_noconv=True, history=0):
        """b, x: fp64 torch CUDA tensors or numpy arrays (host). x is updated.
        history=K > 0 records the first K iterations (ndiag_set_history) into
        info["history"], an array of shape (min(iters, K), 4)."""
        info = SolveInfo()
        hist = None
        if history:
            hist = np.zeros((int(history), 4))
            _check(self.L, self.L.ndiag_set_history(self.h, hist.ctypes.data, int(history)))
        try:
            st = self.L.krylov_solve(self.h, method, precond, mode, _ptr(_omega(omega, self.dim)), float(rtol),
                                     int(maxit), _ptr(b), _ptr(x), ctypes.byref(info))
        finally:
            if hist is not None:
                self.L.ndiag_set_history(self.h, None, 0)
        if st != OK and (raise_on_noconv or st != ENOCONV):
            _check(self.L, st)
        out = dict(iters=info.iterations, outer=info.outer, relres=info.relres, seconds=info.seconds,
                   status=STATUS_NAMES[st])
        if hist is not None:
            out["history"] = hist[: min(info.iterations, int(history))].copy()
        return out


    def tune_omega(self, b, rtol=1e-8, maxit=20000, budget=60, omega=1.0):
        """Per-direction relaxation factors for the stationary decomposed SOR
        iteration (coordinate search on the GPU). Returns (factors, sweeps)."""
        om = _omega(omega, self.dim).copy()
        its = ctypes.c_int(0)
        st = self.L.ndiag_tune_omega(self.h, _ptr(b), float(rtol), int(maxit), int(budget), _ptr(om),
                                     ctypes.byref(its))
        _check(self.L, st)
        return [float(v) for v in om[: 1 << self.dim]], its.value


class Batch:
    """Many independent 2D 5-point problems solved together (fp32 SSOR-PCG with
    fp64 refinement). problems: list of dicts with n=(nx, ny, 1) and diags
    (5 x nx*ny); vectors are concatenated in problem order."""

    def __init__(self, problems, tile=None, omega=1.0, stream=None):
        import torch
        self.L = load()
        _install_torch_allocator(self.L)
        self.count = len(problems)
        nx = np.array([int(p["n"][0]) for p in problems], dtype=np.int64)
        ny = np.array([int(p["n"][1]) for p in problems], dtype=np.int64)
        self._diags = [np.ascontiguousarray(p["diags"], dtype=np.float64) for p in problems]
        ptrs = (ctypes.c_void_p * self.count)(*[d.ctypes.data for d in self._diags])
        tl = None if tile is None else np.ascontiguousarray(
            np.broadcast_to(np.asarray(tile, dtype=np.int32), (self.count,)))
        self.offsets = np.concatenate([[0], np.cumsum(nx * ny)]).astype(np.int64)
        s = stream if stream is not None else torch.cuda.current_stream().cuda_stream
        h = ctypes.c_void_p()
        _check(self.L, self.L.ndiag_batch_create(ctypes.byref(h), self.count, _ptr(nx), _ptr(ny), ptrs,
                                                 _ptr(tl), float(omega), ctypes.c_void_p(s)))
        self.h = h

    @property
    def cells(self):
        return int(self.L.ndiag_batch_cells(self.h))

    def launches(self):
        return int(self.L.ndiag_batch_launches(self.h))

    def autotune(self, b):
        _check(self.L, self.L.ndiag_batch_autotune(self.h, _ptr(b)))

    def tiles(self):
        t = np.zeros(self.count, dtype=np.int32)
        _check(self.L, self.L.ndiag_batch_tiles(self.h, _ptr(t)))
        return t

    def ssor_apply(self, r, z):
        """z = M^-1 r for every problem (the batch's decomposed SSOR, fp32);
        r, z: concatenated float32 CUDA tensors."""
        _check(self.L, self.L.ndiag_batch_ssor_apply(self.h, _ptr(r), _ptr(z)))

    def solve(self, b, x, rtol=1e-8, maxit=20000, raise_on_noconv=True):
        """b, x: concatenated fp64 CUDA tensors; x is updated. Returns per-problem infos."""
        infos = (SolveInfo * self.count)()
        st = self.L.ndiag_batch_solve(self.h, float(rtol), int(maxit), _ptr(b), _ptr(x), infos)
        if st != OK and (raise_on_noconv or st != ENOCONV):
            _check(self.L, st)
        return [dict(iters=i.iterations, outer=i.outer, relres=i.relres, seconds=i.seconds,
                     status=STATUS_NAMES[i.status] if 0 <= i.status < len(STATUS_NAMES) else str(i.status))
                for i in infos]

    def close(self):
        if getattr(self, "h", None):
            self.L.ndiag_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


PRECISIONS = {"fp64": 0, "fp32": 1, "fp32_d16": 2}


class Server:
    """Continuous-batching solve server: submit() queues a request, poll() /
    wait() collect the result. Requests run concurrently in `slots` workers,
    admitted when a slot is free and their memory fits the budget."""

    def __init__(self, slots=4, mem_budget=0):
        self.L = load()
        h = ctypes.c_void_p()
        _check(self.L, self.L.ndiag_server_create(ctypes.byref(h), int(slots), int(mem_budget)))
        self.h = h
        self._sizes = {}

    def submit(self, problem, method=PCG, precond=PREC_SSOR, precision="fp64", rtol=1e-8, maxit=20000,
               omega=1.0):
        dim = int(problem["dim"])
        n = list(problem["n"]) + [1, 1, 1]
        sub = list(problem.get("sub", (1, 1, 1))) + [1, 1, 1]
        diags = np.ascontiguousarray(problem["diags"], dtype=np.float64)
        b = np.ascontiguousarray(problem["b"], dtype=np.float64)
        r = Request(dim, int(problem["stencil"]), (ctypes.c_int64 * 3)(*n[:3]), (ctypes.c_int * 3)(*sub[:3]),
                    diags.ctypes.data, b.ctypes.data, int(method), int(precond), PRECISIONS[precision],
                    float(rtol), int(maxit), float(omega))
        t = ctypes.c_uint64()
        _check(self.L, self.L.serve_submit(self.h, ctypes.byref(r), ctypes.byref(t)))
        self._sizes[t.value] = b.size
        return t.value

    def poll(self, ticket):
        """None while pending, else (result dict, x as numpy)."""
        res = Result()
        x = np.empty(self._sizes[ticket])
        st = self.L.serve_poll(self.h, ctypes.c_uint64(ticket), ctypes.byref(res), x.ctypes.data_as(ctypes.c_void_p))
        if st == EBUSY:
            return None
        _check(self.L, st)
        del self._sizes[ticket]
        i = res.info
        return (dict(status=STATUS_NAMES[res.status], iters=i.iterations, outer=i.outer, relres=i.relres,
                     queue_s=res.queue_s, run_s=res.run_s, latency_s=res.latency_s, cells=res.cells), x)

    def wait(self, ticket, timeout=600.0):
        st = self.L.ndiag_server_wait(self.h, ctypes.c_uint64(ticket), float(timeout))
        if st not in (OK, EBUSY):
            _check(self.L, st)
        return self.poll(ticket) if st == OK else None

    def stats(self):
        s = ServerStats()
        _check(self.L, self.L.ndiag_server_stats(self.h, ctypes.byref(s)))
        return dict(queued=s.queued, running=s.running, max_running=s.max_running, solved=s.solved,
                    budget_bytes=s.budget_bytes, in_use_bytes=s.in_use_bytes)

    def close(self):
        if getattr(self, "h", None):
            self.L.ndiag_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Eikonal:
    """Decomposed fast sweeping for |grad u| = f on an nx x ny grid of spacing
    h, resident on the current CUDA device (fp64)."""

    def __init__(self, n, h, f, sub=(1, 1), stream=None):
        import torch
        self.L = load()
        _install_torch_allocator(self.L)
        self.n = (int(n[0]), int(n[1]))
        self.N = self.n[0] * self.n[1]
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        fa = np.ascontiguousarray(f, dtype=np.float64).reshape(self.N)
        n64 = np.array(self.n, dtype=np.int64)
        sub32 = np.array(list(sub)[:2], dtype=np.int32)
        h_ = ctypes.c_void_p()
        _check(self.L, self.L.eikonal_create(ctypes.byref(h_), _ptr(n64), float(h), _ptr(fa), _ptr(sub32),
                                             ctypes.c_void_p(self.stream.cuda_stream)))
        self.h = h_

    def close(self):
        if getattr(self, "h", None):
            self.L.eikonal_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sweep(self, t, u_old, u_new, wait=True):
        """One sweep at phase t (device tensors); returns the largest change if wait."""
        ch = ctypes.c_double()
        _check(self.L, self.L.eikonal_sweep(self.h, int(t), _ptr(u_old), _ptr(u_new),
                                            ctypes.byref(ch) if wait else None))
        return ch.value if wait else None

    def solve(self, u, delta=0.0, max_rounds=1000, raise_on_noconv=True):
        """u: fp64 device tensor or host array, start values in, result out."""
        info = EikInfo()
        st = self.L.eikonal_solve(self.h, _ptr(u), float(delta), int(max_rounds), ctypes.byref(info))
        if st != OK and (raise_on_noconv or st != ENOCONV):
            _check(self.L, st)
        return dict(sweeps=info.sweeps, converged=bool(info.converged), change=info.change,
                    seconds=info.seconds, launches=info.launches, status=STATUS_NAMES[st])
