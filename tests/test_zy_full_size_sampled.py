"""The benchmark workload at its full size, in the configurations bench.py times,
against stored oracle values (runs last: the longest GPU test).

Four layers (interfaces z = 0, -1, -2, k = (1, 1.5, 2, 2.5) + 0.02i), N = 2^20
points in 64 Gaussian clusters, p = 12, depth 6, theta 0.5, complex64 currents
(the workload's own type).  J is kept on ~1400 sources -- 400 random ones and
the 8 nearest points of every target, so that near-field pairs are in the sum --
and the oracle's direct FP64 sum over them is evaluated at 128 targets, half of
them within 0.1 of an interface.  Err_2 of Section 4 over the targets must meet
the 1e-6 bar of the metric and Err_max 1e-5, for the mixed form with M2L, M2M
and L2L on the tensor cores (tensor_cores = 3) and for the FP64 form."""
import numpy as np
import pytest

import oracle_refs as R
from paper_2507_18491_gb300 import lmfmm

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def sample():
    return R.reference("four_layer_n1048576")


@pytest.mark.parametrize("precision,tensor_cores,kernel", [("mixed", 3, 3), ("fp64", 1, 0)])
def test_four_layer_full_size_sampled(sample, precision, tensor_cores, kernel):
    w, tg, src, J, ref = sample
    prec = lmfmm.MIXED if precision == "mixed" else lmfmm.FP64
    op = lmfmm.Operator(w.d, w.k, w.xyz, p=12, depth=6, theta=0.5, precision=prec,
                        tensor_cores=tensor_cores).build()
    try:
        got = op.matvec(torch.from_numpy(J.astype(np.complex64)).cuda())
        op.check()
        got = got.cpu().numpy().astype(np.complex128)
        st = op.stats()
    finally:
        op.close()
    e2, em = R.err2(got[tg], ref), R.errmax(got[tg], ref)
    print("%s: Err_2 %.3e Err_max %.3e on %d targets (N = %d, %d sources kept)"
          % (precision, e2, em, tg.size, w.N, src.size))
    assert st["m2l_kernel"] == kernel
    assert e2 < 1e-6 and em < 1e-5
