"""The comparison rules on the GPU (FP64): Gauss-Legendre on every element of
each row's support, and the Newton-Cotes-type weighted rules, through the
same row kernel (its general-points class), against the oracle's assembly
with the same rules: <= 1e-12 relative per matrix."""
import numpy as np
import pytest

import oracle
from paper_1710_01048_gb300 import binding as wq
from paper_1710_01048_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12


def check(A, O, what):
    em = np.max(np.abs(A - O)) / np.max(np.abs(O))
    ef = np.linalg.norm(A - O) / np.linalg.norm(O)
    assert em <= TOL and ef <= TOL, f"{what}: {em:.3e} {ef:.3e}"


@pytest.mark.parametrize("mode", ["gl", "nc"])
@pytest.mark.parametrize("p", [2, 3])
@pytest.mark.parametrize("dim,nel", [(3, (9, 7, 6)), (3, (3, 3, 2)), (3, (1, 1, 1)), (3, (25, 4, 5)), (2, (13, 5)),
                                     (2, (1, 3))])
def test_comparison_rule_parity(mode, p, dim, nel):
    g, c = inputs.make(dim, p, nel, 0.05, "exp", 0.1, seed=6)
    R = wq.Rules(dim, p, nel, rule=mode)
    gd = [torch.from_numpy(x).cuda() for x in g]
    M, K = wq.assemble(R, gd, torch.from_numpy(c).cuda(), "fp64")
    Mo, Ko = oracle.assemble_rule(mode, dim, p, nel, g, c)
    check(M.cpu().numpy(), Mo, f"M {mode}")
    check(K.cpu().numpy(), Ko, f"K {mode}")
    # single matrices and a row range
    Ms, _ = wq.assemble(R, gd, torch.from_numpy(c).cuda(), "fp64", stiffness=False)
    assert torch.equal(Ms, M)
    rb, re = R.rows // 3, R.rows // 3 + max(1, R.rows // 4)
    Mr, Kr = wq.assemble(R, gd, torch.from_numpy(c).cuda(), "fp64", row_begin=rb, row_end=re)
    assert torch.equal(Mr, M[rb:re]) and torch.equal(Kr, K[rb:re])
    R.close()


@pytest.mark.parametrize("mode", ["gl", "nc"])
def test_comparison_rule_benchmark_size_sampled(mode):
    w, g, c = inputs.workload("3d_p3_64")
    p, nel = w["p"], w["nel"]
    R = wq.Rules(3, p, nel, rule=mode)
    gd = [torch.from_numpy(x).cuda() for x in g]
    M, K = wq.assemble(R, gd, torch.from_numpy(c).cuda(), "fp64")
    n1, n12 = nel[0] + p, (nel[0] + p) * (nel[1] + p)
    for rb, re in [(0, 40), (n12 * 30 + n1 * 20, n12 * 30 + n1 * 21), (R.rows - 40, R.rows)]:
        Mo, Ko = oracle.assemble_rule(mode, 3, p, nel, g, c, rb, re)
        check(M[rb:re].cpu().numpy(), Mo, f"M {mode} {rb}")
        check(K[rb:re].cpu().numpy(), Ko, f"K {mode} {rb}")
    R.close()


def test_comparison_rules_reject_other_paths():
    p, nel = 2, (5, 4, 3)
    g, c = inputs.make(3, p, nel, 0.0, "one")
    gd = [torch.from_numpy(x).cuda() for x in g]
    R = wq.Rules(3, p, nel, rule="nc")
    for prec in ("mixed", "df64"):
        with pytest.raises(wq.WqError) as ei:
            wq.assemble(R, gd, torch.from_numpy(c).cuda(), prec)
        assert ei.value.status == wq.WQ_ERR_UNSUPPORTED
    G = torch.zeros((R.rows, R.band), dtype=torch.float64, device="cuda")
    with pytest.raises(wq.WqError) as ei:
        wq.assemble_adjoint(R, gd, G, None, "fp64")
    assert ei.value.status == wq.WQ_ERR_UNSUPPORTED
    R.close()
