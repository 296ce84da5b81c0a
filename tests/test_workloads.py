"""The synthetic inputs follow the stated recipes (CPU): the four-layer clustered
benchmark workload, the two- and three-layer parity workloads and the batch of
many problems (the Section 4 media are checked in test_golden_paper_inputs.py)."""
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


def test_two_layer_recipe():
    """C1: two layers, interface z = 0, k = (0.8, 1.2) real; 512 points uniform
    in [-1,1]^2 x [0.1, 2.1] (all in the upper layer); complex128 currents."""
    w = W.two_layer_small(seed=1001)
    assert w.N == 512 and w.p == 6 and w.depth == 2 and w.dtype == "c128"
    np.testing.assert_array_equal(w.d, [0.0])
    np.testing.assert_array_equal(w.k, [0.8, 1.2])
    lo, hi = w.xyz.min(axis=0), w.xyz.max(axis=0)
    assert np.all(lo >= [-1, -1, 0.1]) and np.all(hi <= [1, 1, 2.1])
    # uniform: each half of every axis holds about half of the points
    for a, mid in enumerate((0.0, 0.0, 1.1)):
        assert abs(np.mean(w.xyz[:, a] < mid) - 0.5) < 0.08


def test_three_layer_recipe():
    """C2: interfaces z = 0, -1.2, k = (0.8, 1.5, 2.0) + 0.01i; N = 65536, half
    uniform in [-1,1]^2 x [0.1, 1.1], half in [-1,1]^2 x [-1.1, -0.1]; p = 10,
    depth 5."""
    w = W.three_layer(seed=1002)
    assert w.N == 65536 and w.p == 10 and w.depth == 5
    np.testing.assert_array_equal(w.d, [0.0, -1.2])
    np.testing.assert_allclose(w.k, np.array([0.8, 1.5, 2.0]) + 0.01j, rtol=0, atol=0)
    up, dn = w.xyz[:32768], w.xyz[32768:]
    assert np.all(up[:, 2] >= 0.1) and np.all(up[:, 2] <= 1.1)
    assert np.all(dn[:, 2] >= -1.1) and np.all(dn[:, 2] <= -0.1)
    assert np.all(np.abs(w.xyz[:, :2]) <= 1.0)
    # currents: i.i.d. N(0, 1) real and imaginary parts
    for part in (w.J.real, w.J.imag):
        assert abs(part.mean()) < 0.01 and abs(part.std() - 1.0) < 0.01


def test_batch_recipe():
    """C4: 64 problems of two or three layers (second interface at -U[0.8, 1.6]),
    k ~ U[0.5, 4] + U[0, 0.02] i per layer, N ~ U[2048, 65536] split evenly over
    the layers, points 0.1 from every interface, complex64 currents."""
    probs = W.batch_problems()
    assert len(probs) == 64
    nl = [w.d.size + 1 for w in probs]
    assert set(nl) == {2, 3}
    for w in probs:
        assert 2048 <= w.N <= 65536 and w.dtype == "c64"
        assert w.d[0] == 0.0 and (w.d.size == 1 or -1.6 <= w.d[1] <= -0.8)
        assert np.all((w.k.real >= 0.5) & (w.k.real <= 4.0) & (w.k.imag >= 0) & (w.k.imag <= 0.02))
        z = w.xyz[:, 2]
        assert np.min(np.abs(z[:, None] - w.d[None, :])) >= 0.1 - 1e-12
        lay = (z[:, None] < w.d[None, :]).sum(axis=1)
        counts = np.bincount(lay, minlength=w.d.size + 1)
        assert counts.max() - counts.min() <= 1
        # complex64 currents, carried in complex128
        np.testing.assert_array_equal(w.J, w.J.astype(np.complex64).astype(np.complex128))
    assert len({w.N for w in probs}) > 50   # uneven sizes
