"""The benchmark workload at its full size, in the configurations bench.py times,
against the oracle on sampled outputs (runs last: the longest GPU test).

Four layers (interfaces z = 0, -1, -2, k = (1, 1.5, 2, 2.5) + 0.02i), N = 2^20
points in 64 Gaussian clusters, p = 12, depth 6, theta 0.55.  J is kept on 400
random sources and zero elsewhere; the oracle's direct FP64 sum over those
sources is evaluated at 16 random targets, and Err_2 of Section 4 over these
targets must meet the 1e-6 bar of the metric, for the mixed form with M2L, M2M
and L2L on the tensor cores (tensor_cores = 3) and for the FP64 form."""
import numpy as np
import pytest

import oracle as O
from paper_2507_18491_gb300 import lmfmm, workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def sample():
    w = W.four_layer_clusters(seed=1005)
    rng = np.random.default_rng(11)
    src = rng.choice(w.N, 400, replace=False)
    tg = rng.choice(w.N, 16, replace=False)
    J = np.zeros_like(w.J)
    J[src] = w.J[src]
    ref, _ = O.direct(w.d, w.k, w.xyz, J, targets=tg, sources=src)
    return w, J, tg, ref


@pytest.mark.parametrize("precision,tensor_cores,kernel", [("mixed", 3, 3), ("fp64", 1, 0)])
def test_four_layer_full_size_sampled(sample, precision, tensor_cores, kernel):
    w, J, tg, ref = sample
    prec = lmfmm.MIXED if precision == "mixed" else lmfmm.FP64
    op = lmfmm.Operator(w.d, w.k, w.xyz, p=12, depth=6, theta=0.55, precision=prec,
                        tensor_cores=tensor_cores).build()
    try:
        got = op.matvec(torch.from_numpy(J).cuda()).cpu().numpy()
        st = op.stats()
    finally:
        op.close()
    err = np.linalg.norm(got[tg] - ref) / np.linalg.norm(ref)
    print("%s: Err_2 %.3e on %d targets (N = %d, %d sources kept)" % (precision, err, tg.size, w.N, 400))
    assert st["m2l_kernel"] == kernel
    assert err < 1e-6
