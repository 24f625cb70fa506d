"""Band-layout helpers for the tests (numpy only; shares nothing with the
CUDA path or the oracle).

Row r = r1 + n1 (r2 + n2 r3) of a band holds (2p+1)^dim entries, offset
index d = d1 + (2p+1) (d2 + (2p+1) d3) with d1 fastest; entry d of row r
belongs to column c_a = r_a - p + d_a in each direction, and columns outside
[0, n_a) hold zeros (the layout of the assembly, Fig. 1)."""
import numpy as np


def band_columns(dim, p, nel):
    """(rows, band) int64 column indices, -1 where the column is outside the mesh."""
    n = [e + p for e in nel]
    nb = 2 * p + 1
    r = np.indices(n[::-1]).reshape(dim, -1)[::-1]  # r[0] fastest over rows
    d = np.indices([nb] * dim).reshape(dim, -1)[::-1]  # d[0] fastest over band entries
    c = r[:, :, None] - p + d[:, None, :]
    ok = np.all((c >= 0) & (c < np.array(n)[:, None, None]), axis=0)
    col = np.zeros(ok.shape, dtype=np.int64)
    stride = 1
    for a in range(dim):
        col += c[a] * stride
        stride *= n[a]
    return np.where(ok, col, -1)


def band_matvec(B, cols, x):
    """y_r = sum over the row's entries of B[r, d] x[cols[r, d]] (FP64)."""
    xs = np.where(cols >= 0, x[np.maximum(cols, 0)], 0.0)
    return np.sum(B.astype(np.float64) * xs, axis=1)


def band_abs_matvec(B, cols, x):
    """sum of |B[r, d]| |x[col]|: the scale a row's matvec error is measured against."""
    xs = np.where(cols >= 0, np.abs(x[np.maximum(cols, 0)]), 0.0)
    return np.sum(np.abs(B.astype(np.float64)) * xs, axis=1)


def band_to_dense(B, cols):
    rows = B.shape[0]
    D = np.zeros((rows, rows))
    r = np.repeat(np.arange(rows), B.shape[1]).reshape(B.shape)
    ok = cols >= 0
    D[r[ok], cols[ok]] = B[ok]
    return D
