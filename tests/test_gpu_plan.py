"""The host-only plan check builds the same structures as lmfmm_build: its
counts of boxes, far pairs, geometries, near pairs and M2L columns equal those
of a built context on the same inputs."""
import pytest

from paper_2507_18491_gb300 import lmfmm
from paper_2507_18491_gb300 import workloads as W


@pytest.mark.gpu
@pytest.mark.parametrize("components", [lmfmm.REACTION, lmfmm.TOTAL])
def test_plan_counts_equal_the_build(components):
    w = W.three_layer(n=4096, seed=1002, p=4)
    opt = dict(p=4, depth=3, theta=0.5)
    rc, info = lmfmm.plan_check(w.d, w.k, w.xyz, components=components, **opt)
    assert rc == lmfmm.OK, info["message"]
    op = lmfmm.Operator(w.d, w.k, w.xyz, precision=lmfmm.FP64, components=components, **opt).build()
    st = op.stats()
    op.close()
    assert st["depth"] == info["depth"]
    assert st["n_boxes"] == info["n_boxes"]
    assert st["n_components"] == info["n_components"]
    assert st["n_m2l_pairs"] == info["n_far_pairs"] + info["n_free_far_pairs"]
    assert st["n_near_pairs"] == info["n_near_pairs"]
    assert st["n_near_point_pairs"] == info["n_near_point_pairs"]
    assert st["n_geometries"] == info["n_geometries"] + info["n_free_geometries"]
    assert st["n_free_geometries"] == info["n_free_geometries"]
    assert st["n_free_near_point_pairs"] == info["n_free_near_point_pairs"]
    assert st["m2l_columns"] == info["n_columns"]
