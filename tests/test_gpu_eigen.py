"""Eigenvalue convergence with the matrices assembled on the GPU (Sec. 4, the
2D and 3D examples): K u = lambda M u on the unit square and cube with
homogeneous Dirichlet conditions, identity map, c = 1, M and K from the
weighted Gaussian rules in FP64 and in double-float (tests/eigen.py).  The error of the 10th
eigenvalue must fall at the rate 2p of the fully integrated Galerkin method
(the paper reports rates close to 2p); the same check runs on the oracle's
matrices in test_oracle_eigen.py."""
import pytest

import eigen
from paper_1710_01048_gb300 import binding as wq
from paper_1710_01048_gb300 import inputs

torch = pytest.importorskip("torch")
pytest.importorskip("scipy.linalg")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp64", "df64"])
@pytest.mark.parametrize("dim,p,meshes", eigen.CASES)
def test_tenth_eigenvalue_converges_at_rate_2p(dim, p, meshes, prec):
    tenth = []
    for n in meshes:
        nel = (n,) * dim
        R = wq.Rules(dim, p, nel)
        gd = [torch.from_numpy(v).cuda() for v in inputs.geometry(p, nel)]
        M, K = wq.assemble(R, gd, None, prec)
        R.close()
        tenth.append(eigen.smallest_ten(dim, p, n, M.cpu().numpy(), K.cpu().numpy())[9])
    errs, rates = eigen.rates(dim, meshes, tenth)
    print(f"{prec} dim {dim} p {p} meshes {meshes} rel. errors {['%.3e' % e for e in errs]} rates "
          f"{['%.2f' % r for r in rates]}")
    assert errs[-1] < errs[0]
    assert 2 * p - 0.6 <= rates[-1] <= 2 * p + 1.0, rates
