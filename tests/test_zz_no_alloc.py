"""lmfmm_direct_noalloc: the all-pairs direct evaluation for callers that
cannot allocate device memory mid-run (their device memory is held by
another allocator, or an allocation must not stall or fail during the
computation).  It must reproduce lmfmm_direct -- same kernels, scratch in a
fixed device array instead of cudaMalloc -- on two calls in a row (the
array keeps the previous call's contents), and reject work beyond its
fixed scratch with an error instead of allocating."""
import numpy as np
import pytest

from paper_2507_18491_gb300 import lmfmm, workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_noalloc_direct_matches_direct_twice():
    rng = np.random.default_rng(31)
    d = np.array([0.0, -1.2])
    k = np.array([0.8, 1.5, 2.0]) + 0.01j
    xyz = W.points_in_layers(rng, d, [40, 40, 40], margin=0.1, xy=0.8)
    op = lmfmm.Operator(d, k, xyz, p=4, depth=1).build()
    for trial in range(2):
        J = torch.from_numpy(W.currents(rng, xyz.shape[0])).cuda()
        ref = op.direct(J).cpu().numpy()
        out = torch.empty_like(J)
        lmfmm.direct_noalloc(op.ctx, J, out)
        got = out.cpu().numpy()
        assert _rel(got, ref) < 1e-12, trial
    op.close()


def test_noalloc_rejects_work_beyond_its_scratch():
    w = W.two_layer_small(n=1200, seed=8)
    op = lmfmm.Operator(w.d, w.k, w.xyz, p=4, depth=1).build()
    J = torch.from_numpy(w.J).cuda()
    out = torch.empty_like(J)
    with pytest.raises(lmfmm.LmfmmError) as ei:
        lmfmm.direct_noalloc(op.ctx, J, out)
    assert ei.value.code == lmfmm.ERR_ARG and "scratch" in str(ei.value)
    op.close()


def test_noalloc_across_contexts_of_different_sizes():
    """The shared array keeps whatever the previous call left: a larger context
    (more leaf pairs and coefficients), then a smaller one with another N and
    depth, then the larger one again must each reproduce lmfmm_direct."""
    rng = np.random.default_rng(41)
    d = np.array([0.0, -1.2])
    k = np.array([0.8, 1.5, 2.0]) + 0.01j
    big = W.points_in_layers(rng, d, [60, 60, 60], margin=0.1, xy=0.8)
    small = W.points_in_layers(rng, d, [25, 0, 30], margin=0.1, xy=0.8)
    ops = {"big": lmfmm.Operator(d, k, big, p=4, depth=1).build(),
           "small": lmfmm.Operator(d, k, small, p=4, depth=2).build()}
    try:
        for name in ("big", "small", "big"):
            op = ops[name]
            J = torch.from_numpy(W.currents(rng, op.N)).cuda()
            ref = op.direct(J).cpu().numpy()
            out = torch.empty_like(J)
            lmfmm.direct_noalloc(op.ctx, J, out)
            assert _rel(out.cpu().numpy(), ref) < 1e-12, name
    finally:
        for op in ops.values():
            op.close()
