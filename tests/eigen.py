"""The Laplace eigenproblem K u = lambda M u of Sec. 4 from band matrices:
homogeneous Dirichlet conditions (the first and last basis function of each
direction removed), the ten smallest eigenvalues by a dense generalized
symmetric solver (scipy).  Exact eigenvalues on the unit square / cube:
pi^2 (i^2 + j^2 [+ k^2]), i, j, k >= 1; the 10th is 17 pi^2 (2D), 11 pi^2 (3D)."""
import numpy as np

from bandops import band_columns

EXACT_10TH = {2: 17 * np.pi ** 2, 3: 11 * np.pi ** 2}
CASES = [(2, 2, (8, 16, 32)), (2, 3, (8, 16, 32)), (3, 2, (4, 8, 12)), (3, 3, (4, 8, 12))]


def smallest_ten(dim, p, nel, M, K):
    import scipy.linalg as sla
    import scipy.sparse as sp

    cols = band_columns(dim, p, (nel,) * dim)
    rows = np.repeat(np.arange(M.shape[0]), M.shape[1]).reshape(M.shape)
    ok = cols >= 0
    n = nel + p
    shape = (M.shape[0],) * 2
    Ms = sp.csr_matrix((M[ok], (rows[ok], cols[ok])), shape=shape)
    Ks = sp.csr_matrix((K[ok], (rows[ok], cols[ok])), shape=shape)
    idx = np.indices((n,) * dim).reshape(dim, -1)[::-1]  # direction 1 fastest, as the rows
    keep = np.nonzero(np.all((idx > 0) & (idx < n - 1), axis=0))[0]
    return sla.eigh(Ks[keep][:, keep].toarray(), Ms[keep][:, keep].toarray(), eigvals_only=True,
                    subset_by_index=[0, 9])


def rates(dim, meshes, tenth):
    errs = [abs(t - EXACT_10TH[dim]) / EXACT_10TH[dim] for t in tenth]
    r = [np.log(errs[i] / errs[i + 1]) / np.log(meshes[i + 1] / meshes[i]) for i in range(len(meshes) - 1)]
    return errs, r
