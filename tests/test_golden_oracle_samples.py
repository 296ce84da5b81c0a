"""The stored oracle values (tests/golden/oracle_*.npz) are the oracle's: a few
entries of every file are recomputed here with the CPU oracle and must agree,
and the inputs they were computed from regenerate identically (CPU)."""
import numpy as np
import pytest

import oracle as O
import oracle_refs as R

S = R.samples


@pytest.mark.parametrize("name", sorted(S.DIRECT))
def test_stored_direct_sums_are_the_oracles(name):
    w, tg, src = S.sample_of(name)
    stored = S.load_direct(name, w, tg, src)
    assert stored is not None, "inputs no longer regenerate the stored sample"
    pick = tg[[0, tg.size // 2, -1]]
    ref, _ = O.direct(w.d, w.k, w.xyz, w.J, targets=pick, sources=src)
    rows = np.searchsorted(tg, pick)
    np.testing.assert_allclose(stored[rows], ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def test_stored_tables_are_the_oracles():
    z = R.tables("tables_p12")
    d, k, p, ix = z["d"], z["k"], int(z["p"]), z["index"]
    l, lp, tu, su, rho, zs, zt = z["geoms"][1]
    ref = O.m2l_table(d, k, int(l), int(lp), int(tu), int(su), 2, 1, p, rho, zs, zt, rtol=1e-12).T
    np.testing.assert_allclose(z["tables"][1, 2], ref[np.ix_(ix, ix)], rtol=1e-12, atol=0)


def test_accuracy_sample_has_near_targets_and_neighbour_sources():
    w, tg, src = S.sample_of("four_layer_n1048576")
    assert tg.size == 128 and np.all(np.isin(tg, src))
    z = w.xyz[tg, 2]
    near = np.min(np.abs(z[:, None] - w.d[None, :]), axis=1) < 0.1
    assert near.sum() >= 64
