"""Tree, far / near lists, M2L geometries and work items of the setup (Sections
3.3 and 3.4.1), built on the host alone and checked by lmfmm_plan_check: every
(component, source leaf, target leaf) pair is reached by exactly one far pair of
an ancestor pair or one near pair (the FMM's split of the double sum), every
index the kernels read is in bounds, every far pair is admissible and carries
its table's geometry.  No GPU; the configurations' own sizes."""
import numpy as np
import pytest

from paper_2507_18491_gb300 import build, lmfmm
from paper_2507_18491_gb300 import workloads as W


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()
    return lmfmm.load()


CASES = {
    "two_layer_n512": (lambda: W.two_layer_small(seed=1001), dict(p=6, depth=2, theta=0.4)),
    "three_layer_n65536": (lambda: W.three_layer(seed=1002), dict(p=10, depth=5, theta=0.45)),
    "four_layer_clusters_n1048576": (lambda: W.four_layer_clusters(seed=1005), dict(p=12, depth=6, theta=0.5)),
    "paper_3layer_m20000": (lambda: W.paper_table_uniform(m=20000, layers=3, seed=1006), dict(p=8, depth=4)),
    "batch_problem_auto_depth": (lambda: W.batch_problems(n_problems=3, seed=1004)[2], dict(p=8, leaf_cap=64)),
}


def layer_of(z, d):
    return np.searchsorted(-np.asarray(d), -z, side="right") if len(d) else np.zeros(z.shape, int)


def expected_leaf_pairs(n_leaves, L):
    """Reaction components of a source layer l and a target layer l' (both
    holding points): one per direction of the wave leaving l (up if an
    interface lies below l, down if one lies above) and per direction of the
    wave arriving in l' (from below if an interface lies below l', from above
    if one lies above); each splits (leaves of l) x (leaves of l')."""
    tot = 0
    for l, a in enumerate(n_leaves):
        for lp, b in enumerate(n_leaves):
            if a and b:
                tot += ((l <= L - 1) + (l >= 1)) * ((lp >= 1) + (lp <= L - 1)) * a * b
    return tot


@pytest.mark.parametrize("name", sorted(CASES))
def test_every_leaf_pair_is_split_exactly_once(name):
    make, opt = CASES[name]
    w = make()
    rc, info = lmfmm.plan_check(w.d, w.k, w.xyz, **opt)
    assert rc == lmfmm.OK, info["message"]
    assert info["n_violations"] == 0 and info["n_components_unchecked"] == 0
    L = w.d.size
    assert info["n_leaf_pairs_checked"] == expected_leaf_pairs(info["n_leaves"], L)
    # nine helical columns per far pair (one for the (sigma5, 0) table, two for
    # each other), cut into work items of at most 64
    assert info["n_columns"] == 9 * info["n_far_pairs"]
    assert info["n_work_items"] >= -(-info["n_columns"] // 64)
    assert info["n_near_pairs"] > 0 and info["n_far_pairs"] > 0
    assert sum(info["n_geometries_level"]) == info["n_geometries"]
    assert 0 < info["max_geometries_component_level"] <= info["n_geometries"]


@pytest.mark.parametrize("name", ["two_layer_n512", "paper_3layer_m20000", "batch_problem_auto_depth"])
def test_leaves_match_an_independent_count(name):
    """Leaves are the occupied cells of side 2 h / 2^depth of the root cell,
    per layer (layer l between interfaces d_{l-1} > z > d_l)."""
    make, opt = CASES[name]
    w = make()
    rc, info = lmfmm.plan_check(w.d, w.k, w.xyz, **opt)
    assert rc == lmfmm.OK, info["message"]
    D, h, c = info["depth"], info["root_half"], np.array(info["root_center"])
    S = 2 * h / 2 ** D
    cells = np.clip(np.floor((w.xyz - (c - h)) / S).astype(np.int64), 0, 2 ** D - 1)
    lay = layer_of(w.xyz[:, 2], w.d)
    want = [len({tuple(v) for v in cells[lay == l]}) for l in range(w.d.size + 1)]
    assert info["n_leaves"] == want
    if opt.get("depth", -1) < 0:   # depth from the leaf cap: fewest levels with <= cap per leaf on average
        nmax = np.bincount(lay).max()
        assert nmax / 8 ** D <= opt["leaf_cap"] < nmax / 8 ** (D - 1)


def test_free_space_lists_split_same_layer_pairs_once():
    w = W.three_layer(n=4096, seed=1002, p=6)
    rc, react = lmfmm.plan_check(w.d, w.k, w.xyz, p=6, depth=4, theta=0.45)
    assert rc == lmfmm.OK
    rc, tot = lmfmm.plan_check(w.d, w.k, w.xyz, p=6, depth=4, theta=0.45, components=lmfmm.TOTAL)
    assert rc == lmfmm.OK, tot["message"]
    n = tot["n_leaves"]
    assert tot["n_free_components"] == sum(1 for a in n if a)
    assert tot["n_leaf_pairs_checked"] == react["n_leaf_pairs_checked"] + sum(a * a for a in n)
    assert tot["n_far_pairs"] == react["n_far_pairs"] and tot["n_free_far_pairs"] > 0
    assert tot["n_columns"] == 9 * (tot["n_far_pairs"] + tot["n_free_far_pairs"])


@pytest.mark.parametrize("flag", [lmfmm.PLAN_DROP_FAR_PAIR, lmfmm.PLAN_DROP_NEAR_PAIR])
def test_a_missing_interaction_is_reported(flag):
    """The hooks remove one pair (ranges and offsets kept consistent): the check
    must see exactly the leaf pairs it carried go missing."""
    w = W.two_layer_small(seed=1001)
    rc, info = lmfmm.plan_check(w.d, w.k, w.xyz, p=6, depth=2, theta=0.4, flags=flag)
    assert rc == lmfmm.ERR_INTERNAL
    assert info["n_violations"] >= 1 and "reached 0 times" in info["message"]


def test_bad_arguments_are_rejected():
    w = W.two_layer_small(seed=1001)
    xyz = w.xyz.copy()
    xyz[5, 2] = w.d[0]
    rc, info = lmfmm.plan_check(w.d, w.k, xyz, p=6, depth=2)
    assert rc == lmfmm.ERR_ARG and "interface" in info["message"]
    rc, info = lmfmm.plan_check(w.d, w.k, w.xyz, p=0, depth=2)
    assert rc == lmfmm.ERR_ARG and "parameter" in info["message"]
    rc, info = lmfmm.plan_check(w.d, w.k, w.xyz, p=6, depth=2, flags=8)
    assert rc == lmfmm.ERR_ARG


def test_depth_tuner_follows_its_cost_terms():
    """With only the near-field term the deepest tree wins (fewest point pairs
    per leaf pair), with only the M2L term the shallowest (fewest far pairs);
    the predictions are the cost model applied to the plan's counts."""
    w = W.three_layer(n=8192, seed=1002, p=6)
    near_only, pn = lmfmm.plan_depth(w.d, w.k, w.xyz, p=6, depths=(2, 3, 4), theta=0.45, unit_ns=(0, 1, 0, 0))
    m2l_only, pm = lmfmm.plan_depth(w.d, w.k, w.xyz, p=6, depths=(2, 3, 4), theta=0.45, unit_ns=(1, 0, 0, 0))
    assert near_only == 4 and m2l_only == 2
    for D in (2, 3, 4):
        rc, info = lmfmm.plan_check(w.d, w.k, w.xyz, p=6, depth=D, theta=0.45)
        assert rc == lmfmm.OK
        assert pn[D] == pytest.approx(info["n_near_point_pairs"] * 1e-6, rel=1e-12)
        assert pm[D] == pytest.approx(info["n_work_items"] * 1e-6, rel=1e-12)


def test_depth_tuner_picks_the_benchmark_depth():
    """With the costs measured on GB300, the four-layer benchmark's tuned leaf
    level is depth 6 (the level its full-size parity test runs)."""
    w = W.four_layer_clusters(seed=1005)
    best, pred = lmfmm.plan_depth(w.d, w.k, w.xyz, p=12, depths=(5, 6, 7), theta=0.5)
    assert best == 6 and min(pred, key=pred.get) == 6
    assert 9.0 < pred[6] < 14.0    # measured: 11.3 ms per matvec at depth 6


def test_degenerate_inputs():
    """One point; one layer (no interface: no reaction component, the free-space
    part only); the root as the only leaf; two points a thousand units apart
    (a root cell far larger than either leaf)."""
    rc, info = lmfmm.plan_check([0.0], [1, 2], [[0.1, 0.2, 0.3]], p=4, depth=2, components=lmfmm.TOTAL)
    assert rc == lmfmm.OK, info["message"]
    assert info["n_leaves"] == [1, 0] and info["n_leaf_pairs_checked"] == 1 + 1   # one reaction, one free
    rng = np.random.default_rng(0)
    x = rng.uniform(-1, 1, (300, 3))
    rc, info = lmfmm.plan_check([], [1.0 + 0j], x, p=4, depth=3, components=lmfmm.TOTAL)
    assert rc == lmfmm.OK and info["n_components"] == 0 and info["n_free_components"] == 1
    assert info["n_leaf_pairs_checked"] == info["n_leaves"][0] ** 2
    rc, info = lmfmm.plan_check([0.0], [1, 2], x, p=4, depth=0, components=lmfmm.TOTAL)
    assert rc == lmfmm.OK and info["n_far_pairs"] == 0 and info["n_free_far_pairs"] == 0
    rc, info = lmfmm.plan_check([0.0], [1, 2], [[0.1, 0.2, 0.3], [1e3, 0, -5]], p=4, depth=4,
                                components=lmfmm.TOTAL)
    assert rc == lmfmm.OK, info["message"]
