"""Writes the stored oracle values under tests/golden/ (oracle_*.npz).

Every value in these files comes from the CPU oracle (``oracle/``) evaluated on
the seeded synthetic inputs of ``paper_2507_18491_gb300.workloads``; nothing is
taken from the GPU library.  The GPU parity tests and the benchmark's accuracy
check read them instead of re-running the slow direct sum; each file also
records checksums of the inputs it was computed from, and a reader that finds
different inputs (another random-number stream) recomputes with the oracle.

    python tests/golden/make_oracle_samples.py [name ...]   # default: all

Cases
  direct sums (Phi_i = sum_j G^r(r_j, r_i) J_j, Section 3.3; Err_2 / Err_max of
  Section 4 are taken over the targets):
    two_layer_n512         all 512 targets, all sources (the two-layer workload)
    three_layer_n65536     256 targets, ~1500 sources (random + nearest neighbours)
    four_layer_n1048576    128 targets, ~1400 sources (random + nearest neighbours)
    three_layer_n4096      64 targets, ~550 sources (tensor-core sweep in p)
    paper_2layer_m1000 /
    paper_3layer_m1000     64 targets, ~700 sources (the Section 4 media, 1000 per layer)
    paper_2layer_m1000000 /
    paper_3layer_m1000000  64 targets, ~700 sources (the same, 10^6 points per layer)
  M2L tables (eq. onedimensionintegral) at p = 12, four-layer medium:
    tables_p12             two geometries, every (sigma, kappa), the (n', nu) blocks of
                           degrees 0-3, 6, 9, 11, 12
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2507_18491_gb300 import workloads as W  # noqa: E402

# name -> (workload factory, sample arguments: n_targets, n_random_sources, n_neighbours, band)
DIRECT = {
    "two_layer_n512": (lambda: W.two_layer_small(), None),
    "three_layer_n65536": (lambda: W.three_layer(), (256, 512, 4, 0.15)),
    "four_layer_n1048576": (lambda: W.four_layer_clusters(), (128, 400, 8, 0.1)),
    "three_layer_n4096": (lambda: W.three_layer(n=4096, p=8, depth=3), (64, 300, 4, 0.15)),
    "paper_2layer_m1000": (lambda: W.paper_table_uniform(m=1000, layers=2), (64, 400, 6, 0.2)),
    "paper_3layer_m1000": (lambda: W.paper_table_uniform(m=1000, layers=3), (64, 400, 6, 0.2)),
    "paper_2layer_m1000000": (lambda: W.paper_table_uniform(m=10 ** 6, layers=2), (64, 400, 6, 0.05)),
    "paper_3layer_m1000000": (lambda: W.paper_table_uniform(m=10 ** 6, layers=3), (64, 400, 6, 0.05)),
}

# four-layer medium of the benchmark; (l, lp, target up, source up, rho, zs, zt) of
# M2L geometries with mapped centre heights: a same-layer component (images across
# the interface above) and a component between neighbouring layers
TABLES = {
    "tables_p12": dict(d=[0.0, -1.0, -2.0], k=[1.0 + 0.02j, 1.5 + 0.02j, 2.0 + 0.02j, 2.5 + 0.02j],
                       p=12, geoms=[(1, 1, 1, 0, 0.3, 0.55, -0.35),
                                    (2, 1, 1, 1, 0.45, -1.2, -0.75)]),
}
SIGMA_KAPPA = ((1, 0), (5, 0), (2, 1), (4, 1), (3, 2))


def checksum(w):
    """Input fingerprint: sums of the coordinates and currents and a few values."""
    return np.array([w.xyz.sum(), np.abs(w.xyz).sum(), w.J.real.sum(), w.J.imag.sum(),
                     w.xyz[0, 0], w.xyz[-1, 2], w.J[0, 0].real, w.J[-1, 2].imag])


def sample_of(name):
    make, args = DIRECT[name]
    w = make()
    if args is None:
        tg = np.arange(w.N, dtype=np.int64)
        src = None
    else:
        tg, src = W.accuracy_sample(w, *args)
    return w, tg, src


def sparse_currents(w, src):
    """J kept on the sampled sources, zero elsewhere."""
    if src is None:
        return w.J
    J = np.zeros_like(w.J)
    J[src] = w.J[src]
    return J


def path(name):
    return os.path.join(HERE, "oracle_%s.npz" % name)


def make_direct(name):
    w, tg, src = sample_of(name)
    t0 = time.time()
    ref, calls = O.direct(w.d, w.k, w.xyz, w.J, targets=tg, sources=src)
    dt = time.time() - t0
    np.savez_compressed(path(name), targets=tg, sources=(src if src is not None else np.zeros(0, np.int64)),
                        all_sources=np.array(src is None), phi=ref, checksum=checksum(w),
                        rtol=np.array(1e-10), seconds=np.array(dt))
    print("%s: %d targets x %s sources, %.0f s" % (name, tg.size, "all" if src is None else src.size, dt),
          flush=True)


# degrees whose (n', nu) blocks are stored: low, middle and the top of p = 12
TABLE_DEGREES = (0, 1, 2, 3, 6, 9, 11, 12)


def table_index(p, degrees=TABLE_DEGREES):
    """Flat indices n^2 + n + m of every order of the listed degrees."""
    return np.concatenate([np.arange(n * n, (n + 1) ** 2) for n in degrees if n <= p])


def make_tables(name):
    c = TABLES[name]
    d, k, p = np.array(c["d"]), np.array(c["k"]), c["p"]
    out = []
    ix = table_index(p)
    t0 = time.time()
    for (l, lp, tu, su, rho, zs, zt) in c["geoms"]:
        tabs = [O.m2l_table(d, k, l, lp, tu, su, sig, kap, p, rho, zs, zt, rtol=1e-12).T[np.ix_(ix, ix)]
                for sig, kap in SIGMA_KAPPA]
        out.append(np.stack(tabs))
    # tables[g, t, i, j] = I-hat[row index[i] = (nu, mu), column index[j] = (n', m')]
    np.savez_compressed(path(name), tables=np.stack(out), index=ix, degrees=np.array(TABLE_DEGREES),
                        geoms=np.array(c["geoms"], float), d=d, k=k, p=np.array(p),
                        seconds=np.array(time.time() - t0))
    print("%s: %d geometries, %.0f s" % (name, len(out), time.time() - t0), flush=True)


def load_direct(name, w, tg, src):
    """Stored oracle values for this sample, or None if the inputs differ."""
    f = path(name)
    if not os.path.exists(f):
        return None
    z = np.load(f)
    same = (np.array_equal(z["targets"], tg) and
            (bool(z["all_sources"]) if src is None else np.array_equal(z["sources"], src)) and
            np.allclose(z["checksum"], checksum(w), rtol=1e-13, atol=0))
    return z["phi"] if same else None


def reference(name):
    """(workload, targets, sources, J with only the sources kept, oracle values):
    stored values when the regenerated inputs match, else the oracle now."""
    w, tg, src = sample_of(name)
    ref = load_direct(name, w, tg, src)
    if ref is None:
        ref, _ = O.direct(w.d, w.k, w.xyz, w.J, targets=tg, sources=src)
    return w, tg, src, sparse_currents(w, src), ref


if __name__ == "__main__":
    names = sys.argv[1:] or list(DIRECT) + list(TABLES)
    for n in names:
        if n in DIRECT:
            make_direct(n)
        else:
            make_tables(n)
