"""Batches of layered problems of uneven size and frequency in one graph:
every problem's result equals its own matvec, the merged persistent M2L and
the tuner's choice of work tiles leave the results unchanged, and one problem
meets the oracle at the mixed form's bar."""
import numpy as np
import pytest

import oracle as O
from paper_2507_18491_gb300 import lmfmm, workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_batch_equals_single_matvecs_and_oracle():
    probs = W.batch_problems(n_problems=6, seed=11, n_min=2048, n_max=6000, p=10)
    ops = [lmfmm.Operator(w.d, w.k, w.xyz, p=10, leaf_cap=64, theta=0.45, precision=lmfmm.MIXED,
                          tensor_cores=3).build() for w in probs]
    try:
        Js = [torch.from_numpy(w.J.astype(np.complex64)).cuda() for w in probs]
        single = [op.matvec(J).cpu().numpy() for op, J in zip(ops, Js)]
        b = lmfmm.Batch(ops)
        try:
            info = b.info()
            assert info["merged"] and info["nwork"] > 0
            outs = [torch.empty_like(J) for J in Js]
            for rep in range(2):                 # first call captures, second replays
                b.matvec(Js, outs)
                b.check()
                for o, s in zip(outs, single):
                    assert rel(o.cpu().numpy(), s) < 1e-5
            b.tune()
            info = b.info()
            assert all(t > 0 for t in info["ms_variant"])
            print("tuned variant %d, ms per variant %s" % (info["variant"], info["ms_variant"]))
            b.matvec(Js, outs)
            b.check()
            for o, s in zip(outs, single):
                assert rel(o.cpu().numpy(), s) < 1e-5
            got = outs[0].cpu().numpy().astype(np.complex128)
        finally:
            b.close()
    finally:
        for op in ops:
            op.close()
    w = probs[0]
    rng = np.random.default_rng(0)
    tg = rng.choice(w.N, 24, replace=False)
    ref, _ = O.direct(w.d, w.k, w.xyz, w.J, targets=tg)
    e = rel(got[tg], ref)
    print("batch problem 0 vs oracle: %.3e" % e)
    assert e < 1e-5
