"""The transposed operator (every matvec stage replaced by its exact
transpose, run in reverse order) against the forward matvec: the bilinear
identity y^T (A x) = (A^T y)^T x and the sesquilinear one <y, A x> = <A^H y, x>
hold to rounding whatever the truncation; by reciprocity (the paper's
first-slot sum, G(r,r') = G(r',r)^T) A^T approximates A itself to the FMM's
truncation error."""
import numpy as np
import pytest

from paper_2507_18491_gb300 import lmfmm, workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _op(w, **kw):
    return lmfmm.Operator(w.d, w.k, w.xyz, **kw).build()


@pytest.mark.parametrize("precision,tc,tol", [(lmfmm.FP64, 1, 1e-12), (lmfmm.MIXED, 0, 2e-6)])
def test_transpose_identity(precision, tc, tol):
    w = W.three_layer(n=3000, p=8, depth=3)
    op = _op(w, p=8, depth=3, theta=0.5, precision=precision, tensor_cores=tc)
    try:
        assert op.stats()["adjoint_transposed"] == 1
        rng = np.random.default_rng(2)
        x = torch.from_numpy(W.currents(rng, w.N)).cuda()
        y = torch.from_numpy(W.currents(rng, w.N)).cuda()
        Ax, Aty, Ahy = op.matvec(x), op.tmatvec(y), op.rmatvec(y)
        op.check()
        assert op.stats()["n_near_point_pairs"] > 0
    finally:
        op.close()
    lhs = torch.sum(y * Ax).item()
    rhs = torch.sum(Aty * x).item()
    assert abs(lhs - rhs) < tol * abs(lhs), (lhs, rhs)
    lhs = torch.vdot(y.flatten(), Ax.flatten()).item()
    rhs = torch.vdot(Ahy.flatten(), x.flatten()).item()
    assert abs(lhs - rhs) < tol * abs(lhs), (lhs, rhs)


def test_transpose_approximates_the_operator_by_reciprocity():
    w = W.three_layer(n=4096, p=10, depth=3)
    op = _op(w, p=10, depth=3, theta=0.45)
    try:
        J = torch.from_numpy(w.J).cuda()
        a = op.matvec(J).cpu().numpy()
        b = op.tmatvec(J).cpu().numpy()
    finally:
        op.close()
    e = np.linalg.norm(a - b) / np.linalg.norm(a)
    print("A^T J vs A J: %.3e" % e)
    assert e < 1e-6


def test_transpose_unsupported_on_the_tensor_core_forms():
    w = W.two_layer_small(n=300, seed=3)
    op = _op(w, p=6, depth=2, precision=lmfmm.MIXED, tensor_cores=1)
    try:
        assert op.stats()["adjoint_transposed"] == 0
        with pytest.raises(lmfmm.LmfmmError) as ei:
            op.tmatvec(torch.from_numpy(w.J).cuda())
        assert ei.value.code == lmfmm.ERR_UNSUPPORTED
    finally:
        op.close()
