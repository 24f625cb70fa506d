"""Pins of the definition the apply and load-vector parity tests use: the
band matvec of the oracle's bands (tests/bandops.py), y = M x and y = K x,
and b = M(f) 1 for the load vector of Eq. Load.

* the column map: for a constant coefficient on the identity map the
  assembled M and K are symmetric (Eq. Mass and Eq. Stiffness are symmetric
  forms, and the weighted rules are exact there, Remark closing Sec. 3), so
  the dense matrices built through the map must be symmetric; a planted
  mistake in the map (the band offsets read with the slowest direction
  first) breaks that;
* the matvec equals the dense product;
* the load vector for f = 1 on the identity map: b_r = integral of B_r =
  prod_a (t_{r_a+p+1} - t_{r_a}) / (p+1) on the open uniform knots (Sec. 2),
  and the entries sum to the domain's volume, 1;
* K 1 = 0 for any coefficient and separable map (the basis is a partition of
  unity, so the gradients of the columns sum to zero).
"""
import numpy as np
import pytest

import oracle
from bandops import band_columns, band_matvec, band_to_dense
from paper_1710_01048_gb300 import inputs

CASES = [(2, 3, (5, 4)), (2, 2, (3, 6)), (3, 2, (3, 2, 4)), (3, 3, (2, 3, 2))]


def knots(p, nel):
    return np.concatenate([np.zeros(p), np.linspace(0.0, 1.0, nel + 1), np.ones(p)])


def integral_b(p, nel):
    t = knots(p, nel)
    return np.array([(t[r + p + 1] - t[r]) / (p + 1) for r in range(nel + p)])


def columns_slowest_first(dim, p, nel):
    # the planted mistake: band offset index read with d_dim fastest
    cols = band_columns(dim, p, nel)
    nb = 2 * p + 1
    perm = np.indices([nb] * dim).reshape(dim, -1)  # d[0] slowest here
    idx = sum(perm[a] * nb ** a for a in range(dim))
    return cols[:, idx]


@pytest.mark.parametrize("dim,p,nel", CASES)
def test_column_map_gives_symmetric_constant_coefficient_matrices(dim, p, nel):
    g = inputs.geometry(p, nel)
    M, K, _ = oracle.assemble(dim, p, nel, g)
    cols = band_columns(dim, p, nel)
    for B in (M, K):
        D = band_to_dense(B, cols)
        assert np.max(np.abs(D - D.T)) <= 1e-14 * np.max(np.abs(D))
    # the planted mistake is caught where the directions differ in size
    if len(set(nel)) > 1:
        D = band_to_dense(M, columns_slowest_first(dim, p, nel))
        assert np.max(np.abs(D - D.T)) > 1e-3 * np.max(np.abs(D))


@pytest.mark.parametrize("dim,p,nel", CASES)
def test_matvec_equals_dense_product(dim, p, nel):
    g, c = inputs.make(dim, p, nel, 0.05, "exp", 0.1, seed=3)
    M, K, _ = oracle.assemble(dim, p, nel, g, c)
    cols = band_columns(dim, p, nel)
    x = np.random.default_rng(4).standard_normal(M.shape[0])
    for B in (M, K):
        D = band_to_dense(B, cols)
        y = band_matvec(B, cols, x)
        assert np.max(np.abs(y - D @ x)) <= 1e-14 * np.max(np.abs(D) @ np.abs(x))


@pytest.mark.parametrize("dim,p,nel", CASES)
def test_load_vector_of_unit_source_is_the_basis_integral(dim, p, nel):
    g = inputs.geometry(p, nel)
    M, _, _ = oracle.assemble(dim, p, nel, g)
    cols = band_columns(dim, p, nel)
    b = band_matvec(M, cols, np.ones(M.shape[0]))
    ints = [integral_b(p, e) for e in nel]
    expect = ints[0]
    for a in range(1, dim):
        expect = np.multiply.outer(ints[a], expect).reshape(-1)
    assert np.max(np.abs(b - expect)) <= 1e-14 * np.max(expect)
    assert abs(b.sum() - 1.0) <= 1e-13


@pytest.mark.parametrize("dim,p,nel", CASES)
def test_stiffness_annihilates_constants(dim, p, nel):
    g, c = inputs.make(dim, p, nel, 0.05, "exp", 0.1, seed=5)
    _, K, _ = oracle.assemble(dim, p, nel, g, c)
    cols = band_columns(dim, p, nel)
    one = np.ones(K.shape[0])
    y = band_matvec(K, cols, one)
    scale = np.sum(np.abs(K), axis=1)
    assert np.max(np.abs(y) / scale) <= 1e-13
