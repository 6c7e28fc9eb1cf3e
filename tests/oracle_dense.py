"""Independent dense/sparse assembly used to pin the oracle (scipy/numpy only).

Nothing here calls the oracle's arithmetic: the matrices are assembled from
the diagonal-major storage and from the implicit-set masks, and solved with
library routines (scipy.sparse.linalg.spsolve, numpy.linalg.solve).
"""
import numpy as np
import scipy.sparse as sp

from paper_1008_3699_gb300.workloads import STENCIL_OFFSETS


def neighbours(n, stencil):
    """(s, N) array of neighbour indices (-1 outside), natural numbering."""
    nx, ny, nz = n
    N = nx * ny * nz
    idx = np.arange(N)
    x = idx % nx
    y = (idx // nx) % ny
    z = idx // (nx * ny)
    out = np.full((stencil, N), -1, dtype=np.int64)
    for k, (ox, oy, oz) in enumerate(STENCIL_OFFSETS[stencil]):
        xx, yy, zz = x + ox, y + oy, z + oz
        ok = (xx >= 0) & (xx < nx) & (yy >= 0) & (yy < ny) & (zz >= 0) & (zz < nz)
        out[k, ok] = xx[ok] + nx * (yy[ok] + ny * zz[ok])
    return out


def assemble(n, stencil, diags, mask=None, include_diag=True):
    """Sparse matrix of the entries A(i, i+off_k) (k >= 1) selected by
    mask (bool (s, N)), plus the diagonal if include_diag."""
    nb = neighbours(n, stencil)
    N = nb.shape[1]
    rows, cols, vals = [], [], []
    if include_diag:
        rows.append(np.arange(N)); cols.append(np.arange(N)); vals.append(diags[0])
    for k in range(1, stencil):
        sel = nb[k] >= 0
        if mask is not None:
            sel &= mask[k]
        rows.append(np.nonzero(sel)[0]); cols.append(nb[k][sel]); vals.append(diags[k][sel])
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(N, N))


def jmask_bool(jm, stencil):
    return np.array([(jm >> k) & 1 for k in range(stencil)], dtype=bool)


def full_n(n):
    return tuple((list(n) + [1, 1, 1])[:3])
