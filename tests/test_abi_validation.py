"""Host-only checks of the C ABI's argument validation (include/ndiag.h: every
call returns a status and never aborts). Each call here is rejected before
the library touches CUDA, so these run without a GPU: null handles and
pointers, unsupported stencils, bad sizes, subdomain counts, precisions,
non-positive diagonals and mismatched allocator hooks all give NDIAG_EINVAL,
with the message ndiag_last_error() documents where the library sets one, and
every constructor leaves *out NULL."""
import ctypes as C

import numpy as np
import pytest

EINVAL = 1
P = C.c_void_p


@pytest.fixture(scope="module")
def lib():
    from paper_1008_3699_gb300 import build
    L = C.CDLL(build.build())
    L.ndiag_last_error.restype = C.c_char_p
    L.ndiag_cells.restype = C.c_int64
    L.ndiag_cells.argtypes = [P]
    L.ndiag_precision.argtypes = [P]
    L.ndiag_mg_levels.argtypes = [P]
    L.ndiag_batch_cells.restype = C.c_int64
    L.ndiag_batch_cells.argtypes = [P]
    L.ndiag_batch_launches.restype = C.c_int64
    L.ndiag_batch_launches.argtypes = [P]
    L.ndiag_create.argtypes = [C.POINTER(P), C.c_int, P, C.c_int, P, P, C.c_int, P]
    L.eikonal_create.argtypes = [C.POINTER(P), P, C.c_double, P, P, P]
    return L


def _create(lib, dim, n, stencil, sub, precision=0, diag=None):
    N = int(np.prod(n[:dim]))
    d = np.full((stencil, N), -0.1)
    d[0] = 1.0 if diag is None else diag
    nn = (C.c_int64 * 3)(*(list(n) + [1, 1, 1])[:3])
    ss = (C.c_int * 3)(*(list(sub) + [1, 1, 1])[:3])
    out = P(12345)
    st = lib.ndiag_create(C.byref(out), dim, C.cast(nn, P), stencil, d.ctypes.data, C.cast(ss, P), precision, None)
    return st, out.value


@pytest.mark.parametrize("dim,stencil", [(2, 7), (3, 5), (3, 9), (1, 3), (2, 3), (4, 7)])
def test_create_rejects_unsupported_stencils(lib, dim, stencil):
    st, h = _create(lib, dim, (4, 4, 4), stencil, (1, 1, 1))
    assert st == EINVAL and h is None
    assert lib.ndiag_last_error() == b"unsupported dim/stencil"


@pytest.mark.parametrize("dim,stencil,n,sub", [
    (2, 5, (0, 4), (1, 1)),            # empty axis
    (2, 5, (4, 4), (5, 1)),            # more subdomains than cells
    (2, 9, (4, 4), (1, 0)),            # no subdomain
    (3, 7, ((1 << 20) + 1, 1, 1), (1, 1, 1)),  # axis too long
])
def test_create_rejects_bad_sizes(lib, dim, stencil, n, sub):
    nn = (C.c_int64 * 3)(*(list(n) + [1, 1, 1])[:3])
    ss = (C.c_int * 3)(*(list(sub) + [1, 1, 1])[:3])
    d = np.ones(stencil)  # never read: the sizes are checked first
    out = P(1)
    st = lib.ndiag_create(C.byref(out), dim, C.cast(nn, P), stencil, d.ctypes.data, C.cast(ss, P), 0, None)
    assert st == EINVAL and out.value is None
    assert lib.ndiag_last_error() == b"bad grid size or subdomain count"


def test_create_rejects_grids_beyond_int32_cells(lib):
    nn = (C.c_int64 * 3)(1 << 11, 1 << 10, 1 << 10)
    ss = (C.c_int * 3)(1, 1, 1)
    d = np.ones(7)
    out = P(1)
    st = lib.ndiag_create(C.byref(out), 3, C.cast(nn, P), 7, d.ctypes.data, C.cast(ss, P), 0, None)
    assert st == EINVAL and out.value is None
    assert lib.ndiag_last_error() == b"grid too large (N must fit in int32)"


@pytest.mark.parametrize("bad", [0.0, -1.0, np.nan])
def test_create_rejects_non_positive_diagonals(lib, bad):
    diag = np.ones(12)
    diag[7] = bad
    st, h = _create(lib, 2, (4, 3), 5, (2, 1), diag=diag)
    assert st == EINVAL and h is None
    assert lib.ndiag_last_error() == b"diagonal entries must be positive"


@pytest.mark.parametrize("precision", [-1, 3, 17])
def test_create_rejects_unknown_precisions(lib, precision):
    st, h = _create(lib, 2, (4, 3), 5, (1, 1), precision=precision)
    assert st == EINVAL and h is None


def test_create_rejects_null_pointers(lib):
    nn = (C.c_int64 * 3)(4, 4, 1)
    ss = (C.c_int * 3)(1, 1, 1)
    d = np.ones((5, 16))
    assert lib.ndiag_create(None, 2, C.cast(nn, P), 5, d.ctypes.data, C.cast(ss, P), 0, None) == EINVAL
    for args in ((None, d.ctypes.data, C.cast(ss, P)), (C.cast(nn, P), None, C.cast(ss, P)),
                 (C.cast(nn, P), d.ctypes.data, None)):
        out = P(1)
        assert lib.ndiag_create(C.byref(out), 2, args[0], 5, args[1], args[2], 0, None) == EINVAL
        assert out.value is None  # constructors clear *out before any other check


def test_allocator_hooks_come_in_pairs(lib):
    hook = C.CFUNCTYPE(P, C.c_size_t, P, P)(lambda n, s, c: None)
    assert lib.ndiag_set_allocator(hook, None, None) == EINVAL
    assert lib.ndiag_set_allocator(None, None, None) == 0  # back to the library's own allocation


def test_every_call_rejects_a_null_handle(lib):
    buf = (C.c_double * 8)()
    p = C.cast(buf, P)
    om = (C.c_double * 8)(*([1.0] * 8))
    pom = C.cast(om, P)
    calls = [
        ("sor_sweep", (None, C.c_int(1), pom, C.c_int64(0), p, p, P(C.addressof(buf) + 8))),
        ("ssor_apply", (None, C.c_int(1), C.c_double(1.0), p, P(C.addressof(buf) + 8))),
        ("mg_apply", (None, C.c_double(1.0), p, P(C.addressof(buf) + 8))),
        ("ilu0_factor", (None, C.c_int(1))),
        ("ilu0_apply", (None, p, p)),
        ("ilu0_apply_noalloc", (None, p, p)),
        ("ndiag_residual", (None, p, p, p, p)),
        ("krylov_solve", (None, C.c_int(0), C.c_int(1), C.c_int(1), pom, C.c_double(1e-8), C.c_int(10), p, p,
                          None)),
        ("ndiag_set_history", (None, p, C.c_int(2))),
        ("ndiag_tune_omega", (None, p, C.c_double(1e-8), C.c_int(10), C.c_int(4), pom, p)),
        ("ndiag_profile", (None, C.c_int(1))),
        ("ndiag_read_counters", (None, p)),
        ("ndiag_set_wavefront", (None, C.c_int(1))),
        ("ndiag_selftest_wait", (None,)),
        ("ndiag_batch_autotune", (None, p)),
        ("ndiag_batch_tiles", (None, p)),
        ("ndiag_batch_solve", (None, C.c_double(1e-8), C.c_int(10), p, p, None)),
        ("ndiag_batch_ssor_apply", (None, p, p)),
        ("serve_submit", (None, p, p)),
        ("serve_poll", (None, C.c_uint64(1), p, None)),
        ("ndiag_server_wait", (None, C.c_uint64(1), C.c_double(0.0))),
        ("ndiag_server_stats", (None, p)),
        ("eikonal_sweep", (None, C.c_int64(0), p, P(C.addressof(buf) + 8), None)),
        ("eikonal_solve", (None, p, C.c_double(0.0), C.c_int(1), None)),
    ]
    for name, args in calls:
        assert getattr(lib, name)(*args) == EINVAL, name
    assert lib.ndiag_cells(None) == 0
    assert lib.ndiag_precision(None) == -1
    assert lib.ndiag_mg_levels(None) == 0
    assert lib.ndiag_batch_cells(None) == 0
    assert lib.ndiag_batch_launches(None) == 0
    for name in ("ndiag_destroy", "ndiag_batch_destroy", "ndiag_server_destroy", "eikonal_destroy"):
        getattr(lib, name)(None)  # a no-op


def test_constructors_reject_bad_arguments(lib):
    out = P(1)
    assert lib.ndiag_server_create(C.byref(out), 0, C.c_size_t(0)) == EINVAL and out.value is None
    out = P(1)
    assert lib.ndiag_server_create(C.byref(out), 65, C.c_size_t(0)) == EINVAL and out.value is None
    nx = (C.c_int64 * 1)(8)
    dp = (P * 1)(None)
    out = P(1)
    for count, omega in ((0, 1.0), (1, 0.0), (1, 2.0)):
        st = lib.ndiag_batch_create(C.byref(out), count, C.cast(nx, P), C.cast(nx, P), C.cast(dp, P), None,
                                    C.c_double(omega), None)
        assert st == EINVAL and out.value is None
    f = np.ones(16)
    nn = (C.c_int64 * 2)(4, 4)
    for h, sub in ((0.0, (1, 1)), (-1.0, (1, 1)), (0.25, (5, 1)), (0.25, (1, 0))):
        ss = (C.c_int * 2)(*sub)
        out = P(1)
        st = lib.eikonal_create(C.byref(out), C.cast(nn, P), h, f.ctypes.data, C.cast(ss, P), None)
        assert st == EINVAL and out.value is None, (h, sub)


def test_create_without_a_device_fails_loudly(lib):
    # No CPU fallback: a valid matrix on a machine without a CUDA device is
    # refused with NDIAG_EDEVICE and the CUDA error in ndiag_last_error().
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    st, h = _create(lib, 2, (6, 5), 5, (2, 1))
    assert st == 5 and h is None  # NDIAG_EDEVICE
    assert lib.ndiag_last_error().startswith(b"cudaGetDevice")
