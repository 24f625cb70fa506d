"""The oracle's matrices reproduce the eigenvalue convergence of Sec. 4: the
error of the 10th Dirichlet eigenvalue on the unit square and cube falls at
the rate 2p (tests/eigen.py; the same check runs on the GPU's matrices)."""
import pytest

import eigen
import oracle
from paper_1710_01048_gb300 import inputs

pytest.importorskip("scipy.linalg")


@pytest.mark.parametrize("dim,p,meshes", eigen.CASES)
def test_oracle_tenth_eigenvalue_converges_at_rate_2p(dim, p, meshes):
    tenth = []
    for n in meshes:
        nel = (n,) * dim
        M, K, _ = oracle.assemble(dim, p, nel, inputs.geometry(p, nel))
        tenth.append(eigen.smallest_ten(dim, p, n, M, K)[9])
    errs, rates = eigen.rates(dim, meshes, tenth)
    assert errs[-1] < errs[0]
    assert 2 * p - 0.6 <= rates[-1] <= 2 * p + 1.0, rates
