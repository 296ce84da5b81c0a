"""The synthetic stand-in for the paper's test workloads reproduces the media and
particle boxes the paper prints (Section 4), read from tests/golden/."""
import os

import numpy as np
import pytest

from paper_2507_18491_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_section4_media.txt")


def _golden():
    out = {}
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, val = line.split(":", 1)
            rows = [[float(x) for x in part.split()] for part in val.split(";")]
            out[key.strip()] = rows if len(rows) > 1 else rows[0]
    return out


@pytest.mark.parametrize("layers", [2, 3])
def test_paper_workload_matches_printed_media(layers):
    g = _golden()
    pre = "two_layer" if layers == 2 else "three_layer"
    m = int(g["accuracy_test.particles_per_box"][0])
    w = W.paper_table_uniform(m=m, layers=layers, p=int(g["efficiency_test.p"][0]))
    assert w.p == 8
    np.testing.assert_array_equal(w.d, np.array(g[pre + ".interfaces"]))
    # k_l = omega sqrt(eps_l mu_l)
    eps, omega, mu = np.array(g[pre + ".eps"]), g["omega"][0], g["mu"][0]
    np.testing.assert_allclose(w.k, omega * np.sqrt(eps * mu), rtol=0, atol=1e-15)
    # m points in each unit cube, each cube inside its own layer
    centres = np.array(g[pre + ".box_centres"]).reshape(-1, 3)
    half = 0.5 * g["box_side"][0]
    assert w.xyz.shape == (m * layers, 3)
    for b, c in enumerate(centres):
        pts = w.xyz[b * m:(b + 1) * m]
        assert np.all(np.abs(pts - c) <= half)
        top = np.inf if b == 0 else w.d[b - 1]
        bot = -np.inf if b == layers - 1 else w.d[b]
        assert np.all((pts[:, 2] < top) & (pts[:, 2] > bot))
