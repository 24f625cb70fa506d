"""Band -> CSR conversion (wq_band_to_csr) against a CSR built on the host
from the band and its column mask."""
import numpy as np
import pytest

from paper_1710_01048_gb300 import binding as wq
from paper_1710_01048_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def host_csr(band, nel, p, rb, re):
    dim = len(nel)
    n = [v + p for v in nel]
    nb = 2 * p + 1
    mask = inputs.band_mask(nel, p)[rb:re] > 0
    # column offset of band entry j: d1 + n1*d2 + n1*n2*d3
    d = np.stack(np.meshgrid(*[np.arange(-p, p + 1)] * dim, indexing="ij"), -1).reshape(-1, dim)[:, ::-1]
    off = np.zeros(nb ** dim, dtype=np.int64)
    stride = 1
    for a in range(dim):
        off += d[:, a] * stride
        stride *= n[a]
    cols = np.arange(rb, re)[:, None] + off[None, :]
    rowptr = np.concatenate([[0], np.cumsum(mask.sum(1))])
    return rowptr, cols[mask], band[mask]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("dim,p,nel", [(3, 3, (9, 6, 5)), (3, 2, (1, 2, 1)), (2, 3, (13, 4)), (3, 3, (20, 3, 7))])
def test_csr_matches_host(dim, p, nel, prec):
    g, c = inputs.make(dim, p, nel, 0.05, "exp", 0.1, seed=1)
    R = wq.Rules(dim, p, nel)
    gd = [torch.from_numpy(x).cuda() for x in g]
    M, K = wq.assemble(R, gd, torch.from_numpy(c).cuda(), prec)
    rng = np.random.default_rng(2)
    ranges = [(0, R.rows)] + [tuple(sorted(rng.integers(0, R.rows + 1, 2))) for _ in range(4)]
    for rb, re in ranges:
        rb, re = int(rb), int(re)
        band = K[rb:re].contiguous()
        rowptr, col, val = wq.band_to_csr(R, band, prec, rb, re)
        hr, hc, hv = host_csr(band.cpu().numpy(), nel, p, rb, re)
        assert np.array_equal(rowptr.cpu().numpy(), hr)
        assert np.array_equal(col.cpu().numpy(), hc)
        assert np.array_equal(val.cpu().numpy(), hv)
        if re > rb:
            # columns increase within each row
            hcol = hc.astype(np.int64)
            for r in range(re - rb):
                seg = hcol[hr[r]:hr[r + 1]]
                assert np.all(np.diff(seg) > 0)
    # the full matrix as a torch sparse CSR tensor reproduces K @ x
    rowptr, col, val = wq.band_to_csr(R, K, prec)
    S = torch.sparse_csr_tensor(rowptr, col.long(), val, size=(R.rows, R.rows))
    x = torch.randn(R.rows, dtype=val.dtype, device="cuda")
    y = S @ x
    # band product: y_r = sum_j K[r, j] x[r + off_j] over valid entries
    hr, hc, hv = host_csr(K.cpu().numpy(), nel, p, 0, R.rows)
    yh = np.zeros(R.rows)
    np.add.at(yh, np.repeat(np.arange(R.rows), np.diff(hr)), hv.astype(np.float64) * x.cpu().numpy()[hc])
    tol = 1e-12 if prec == "fp64" else 1e-4
    assert np.max(np.abs(y.cpu().numpy() - yh)) <= tol * np.max(np.abs(yh))
    R.close()
