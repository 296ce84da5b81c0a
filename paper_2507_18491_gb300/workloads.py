"""Seeded synthetic workloads for the layered-media Maxwell FMM.

This module holds only input generators: layer stacks, point clouds and
current densities.  It contains none of the method's arithmetic, so both the
CUDA path and the CPU oracle may draw their inputs from it.

The paper's own experiments (Section 4) use uniform random particles in unit
cubes inside each layer; every workload here is synthetic in the same spirit.
Media are given by interface heights ``d`` (strictly decreasing) and layer
wavenumbers ``k`` (Im k >= 0), with mu = 1 and omega = 1 throughout, so that
eps_l = k_l**2 (Section 3.1, eq. for k_l).
"""
from __future__ import annotations

import dataclasses
import numpy as np


@dataclasses.dataclass
class Workload:
    name: str
    d: np.ndarray            # [L] interface heights, strictly decreasing
    k: np.ndarray            # [L+1] complex layer wavenumbers
    xyz: np.ndarray          # [N, 3] float64 point coordinates
    J: np.ndarray            # [N, 3] complex128 current densities
    p: int                   # truncation order
    depth: int               # octree depth (0 = root only)
    dtype: str               # "c128" or "c64": the precision J is drawn in

    @property
    def N(self) -> int:
        return int(self.xyz.shape[0])


def _currents(rng, n, c64):
    J = rng.standard_normal((n, 3)) + 1j * rng.standard_normal((n, 3))
    if c64:
        J = J.astype(np.complex64).astype(np.complex128)
    return J


def _uniform_box(rng, n, lo, hi):
    lo = np.asarray(lo, float)
    hi = np.asarray(hi, float)
    return lo + (hi - lo) * rng.random((n, 3))


def two_layer_small(n=512, seed=1001):
    """Two layers, interface z=0, k=(0.8, 1.2); points in the upper layer."""
    rng = np.random.default_rng(seed)
    xyz = _uniform_box(rng, n, (-1, -1, 0.1), (1, 1, 2.1))
    return Workload("two_layer_n%d" % n, np.array([0.0]),
                    np.array([0.8, 1.2], dtype=complex), xyz,
                    _currents(rng, n, False), p=6, depth=2, dtype="c128")


def three_layer(n=65536, seed=1002, p=10, depth=5):
    """Three layers, interfaces z=0,-1.2, k=(0.8,1.5,2.0)+0.01i.

    Half the points are uniform in [-1,1]^2 x [0.1,1.1] (layer 0), half in
    [-1,1]^2 x [-1.1,-0.1] (layer 1)."""
    rng = np.random.default_rng(seed)
    n0 = n // 2
    xyz = np.concatenate([
        _uniform_box(rng, n0, (-1, -1, 0.1), (1, 1, 1.1)),
        _uniform_box(rng, n - n0, (-1, -1, -1.1), (1, 1, -0.1)),
    ])
    return Workload("three_layer_n%d" % n, np.array([0.0, -1.2]),
                    np.array([0.8, 1.5, 2.0]) + 0.01j, xyz,
                    _currents(rng, n, False), p=p, depth=depth, dtype="c128")


def four_layer_clusters(n=1 << 20, seed=1005, p=12, depth=None, nclusters=64,
                        sigma=0.05):
    """Four layers, interfaces z=0,-1,-2, k=(1,1.5,2,2.5)+0.02i.

    ``nclusters`` Gaussian clusters (std ``sigma``), half in layer 1
    (-1<z<0) and half in layer 2 (-2<z<-1).  Cluster centres are uniform in
    [-1,1]^2 x (layer shrunk by 0.2 on each side).  Points closer than 0.01
    to an interface, or outside their cluster's layer, are redrawn."""
    rng = np.random.default_rng(seed)
    d = np.array([0.0, -1.0, -2.0])
    per = n // nclusters
    pts = []
    for c in range(nclusters):
        top, bot = (0.0, -1.0) if c < nclusters // 2 else (-1.0, -2.0)
        cen = np.array([rng.uniform(-1, 1), rng.uniform(-1, 1),
                        rng.uniform(bot + 0.2, top - 0.2)])
        m = per if c < nclusters - 1 else n - per * (nclusters - 1)
        got = np.empty((0, 3))
        while got.shape[0] < m:
            q = cen + sigma * rng.standard_normal((2 * m, 3))
            ok = (q[:, 2] < top - 0.01) & (q[:, 2] > bot + 0.01)
            got = np.concatenate([got, q[ok]])
        pts.append(got[:m])
    xyz = np.concatenate(pts)
    if depth is None:
        depth = 6
    return Workload("four_layer_clusters_n%d" % n, d,
                    np.array([1.0, 1.5, 2.0, 2.5]) + 0.02j, xyz,
                    _currents(rng, n, True), p=p, depth=depth, dtype="c64")


def paper_table_uniform(m=1000, layers=2, seed=1006, p=8, depth=3):
    """The efficiency-test workload of Section 4: m uniform points per layer
    in unit cubes centred at (0.5,0.5,0.75), (0.5,0.5,-0.75)[, (0.5,0.5,-2.25)],
    omega=2, mu=1, eps=(1.2,0.8[,1.3]) so k=2*sqrt(eps)."""
    rng = np.random.default_rng(seed)
    if layers == 2:
        d = np.array([0.0])
        eps = np.array([1.2, 0.8])
        cz = [0.75, -0.75]
    else:
        d = np.array([0.0, -1.5])
        eps = np.array([1.2, 0.8, 1.3])
        cz = [0.75, -0.75, -2.25]
    xyz = np.concatenate([
        _uniform_box(rng, m, (0, 0, z - 0.5), (1, 1, z + 0.5)) for z in cz])
    k = (2.0 * np.sqrt(eps)).astype(complex)
    return Workload("paper_table_%dlayer_m%d" % (layers, m), d, k, xyz,
                    _currents(rng, xyz.shape[0], False), p=p, depth=depth,
                    dtype="c128")


def random_stack(rng, n_layers, lossy=True):
    """A random admissible stack for small property tests."""
    t = rng.uniform(0.6, 1.4, max(n_layers - 2, 0))
    d = np.concatenate([[0.0], -np.cumsum(t)]) if n_layers > 1 else np.zeros(0)
    k =rng.uniform(0.6, 2.5, n_layers) + (1j * rng.uniform(0.0, 0.05, n_layers)
                                           if lossy else 0.0)
    return d, k.astype(complex)


def points_in_layers(rng, d, counts, margin=0.1, xy=1.0, height=1.0):
    """Uniform points in each listed layer, ``margin`` away from interfaces.

    counts[l] points in layer l; unbounded top/bottom layers are cut to
    ``height``."""
    d = np.asarray(d, float)
    L = d.size
    out = []
    for l, c in enumerate(counts):
        if c == 0:
            continue
        top = d[l - 1] if l >= 1 else (d[0] + height if L else height)
        bot = d[l] if l < L else d[L - 1] - height
        out.append(_uniform_box(rng, c, (-xy, -xy, bot + margin),
                                (xy, xy, top - margin)))
    return np.concatenate(out) if out else np.zeros((0, 3))


def currents(rng, n):
    return _currents(rng, n, False)


def accuracy_sample(w, n_targets, n_random_sources, n_neighbours, band, seed=11,
                    near_fraction=0.5):
    """Seeded target and source subsets for checking a matvec against a direct
    sum (Err_2 / Err_max of Section 4 over the targets).

    Half of the targets (``near_fraction``) are drawn among the points closer
    than ``band`` to an interface, where the images of nearby sources fall next
    to the targets and the near-field (direct) sums of the FMM are exercised;
    the rest uniformly.  The sources are ``n_random_sources`` uniform draws plus
    the ``n_neighbours`` nearest points of every target (itself included, so
    the self term is in the sum).  Returns sorted unique index arrays
    (targets, sources)."""
    rng = np.random.default_rng(seed)
    z = w.xyz[:, 2]
    dist = np.min(np.abs(z[:, None] - np.asarray(w.d, float)[None, :]), axis=1) \
        if np.asarray(w.d).size else np.full(w.N, np.inf)
    close = np.flatnonzero(dist < band)
    n_near = min(int(round(near_fraction * n_targets)), close.size)
    tg_near = rng.choice(close, n_near, replace=False) if n_near else np.zeros(0, np.int64)
    rest = np.setdiff1d(np.arange(w.N), tg_near)
    tg_far = rng.choice(rest, n_targets - n_near, replace=False)
    targets = np.unique(np.concatenate([tg_near, tg_far])).astype(np.int64)
    src = [rng.choice(w.N, min(n_random_sources, w.N), replace=False)]
    for t in targets:
        d2 = np.sum((w.xyz - w.xyz[t]) ** 2, axis=1)
        src.append(np.argpartition(d2, n_neighbours)[:n_neighbours] if n_neighbours < w.N
                   else np.arange(w.N))
        src.append(np.array([t]))
    sources = np.unique(np.concatenate(src)).astype(np.int64)
    return targets, sources


def batch_problems(n_problems=64, seed=1004, n_min=2048, n_max=65536, k_min=0.5, k_max=4.0, p=8):
    """Many layered problems of uneven size and frequency (the batched
    configuration): each has two or three layers (interfaces z = 0 and, for
    three, a second one at -U[0.8, 1.6]), layer wavenumbers U[k_min, k_max]
    with a small loss U[0, 0.02] i, N ~ U[n_min, n_max] points split evenly
    over the layers (uniform in [-1,1]^2 x each layer, 0.1 from interfaces,
    unbounded layers cut at height 1) and complex64 currents."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n_problems):
        nl = int(rng.integers(2, 4))
        d = np.array([0.0]) if nl == 2 else np.array([0.0, -rng.uniform(0.8, 1.6)])
        k = rng.uniform(k_min, k_max, nl) + 1j * rng.uniform(0.0, 0.02, nl)
        n = int(rng.integers(n_min, n_max + 1))
        counts = [n // nl + (1 if j < n % nl else 0) for j in range(nl)]
        xyz = points_in_layers(rng, d, counts, margin=0.1, xy=1.0, height=1.0)
        out.append(Workload("batch_%d_n%d" % (i, n), d, k.astype(complex), xyz,
                            _currents(rng, n, True), p=p, depth=-1, dtype="c64"))
    return out
