"""The synthetic inputs follow the stated recipe (CPU): the four-layer clustered
benchmark workload and the three-layer parity workload."""
import numpy as np

from paper_2507_18491_gb300 import workloads as W


def test_four_layer_clusters_recipe():
    w = W.four_layer_clusters(n=1 << 16, seed=1005)
    assert w.N == 1 << 16 and w.p == 12
    np.testing.assert_array_equal(w.d, [0.0, -1.0, -2.0])
    np.testing.assert_allclose(w.k, np.array([1.0, 1.5, 2.0, 2.5]) + 0.02j, rtol=0, atol=0)
    z = w.xyz[:, 2]
    # layers 1 and 2 only, at least 0.01 away from every interface
    assert np.all((z < 0.0) & (z > -2.0))
    assert np.min(np.abs(z[:, None] - w.d[None, :])) >= 0.01
    # 64 clusters of equal size, the first half in layer 1, the second in layer 2
    per = w.N // 64
    for c in range(64):
        zc = z[c * per:(c + 1) * per]
        if c < 32:
            assert np.all(zc > -1.0)
        else:
            assert np.all(zc < -1.0)
        # Gaussian clusters of standard deviation 0.05
        s = w.xyz[c * per:(c + 1) * per].std(axis=0)
        assert np.all(s < 0.06) and np.all(s > 0.03)
    assert w.J.shape == (w.N, 3) and np.iscomplexobj(w.J)


def test_workloads_are_seeded():
    a = W.four_layer_clusters(n=4096, seed=7)
    b = W.four_layer_clusters(n=4096, seed=7)
    c = W.four_layer_clusters(n=4096, seed=8)
    np.testing.assert_array_equal(a.xyz, b.xyz)
    np.testing.assert_array_equal(a.J, b.J)
    assert not np.array_equal(a.xyz, c.xyz)
