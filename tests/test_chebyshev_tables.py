"""The Chebyshev machinery of the M2L tabulation (Section 3.4, Appendices A
and B), exactly as the library's host routines build it, against the oracle's
normalised Legendre functions (its own recurrence with the complex extension
cos b = k_z / k, sin b = k_rho / k): the B-expansion of every P^_n^m, at real
and complex angles, and the product tensor G of a source and a target function
re-expanded in the variable of the smaller wavenumber (Appendix A's C^{ab}
coefficients).  No GPU."""
import numpy as np
import pytest

import oracle
from paper_2507_18491_gb300 import build, lmfmm


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()
    oracle.build()
    return lmfmm.load()


def tau(n, m, c, s):
    if n % 2 == 0 and m % 2 == 0:
        return 1.0 + 0 * c
    if n % 2 == 1 and m % 2 == 0:
        return 1.0 / c
    if n % 2 == 1:
        return s
    return s / c


def cheb(x, K):
    """T_0 .. T_K at a real or complex x (three-term recurrence)."""
    T = [1.0 + 0 * x, x]
    for _ in range(K - 1):
        T.append(2 * x * T[-1] - T[-2])
    return np.array(T[:K + 1])


def f_ref(p, c, s):
    """P^_n^m(c, s) / tau_nm for every (n, m), from the oracle."""
    P = oracle.legendre(p, c, s)
    return np.array([P[n * (n + 1) // 2 + m] / tau(n, m, c, s) for n in range(p + 1) for m in range(n + 1)])


ANGLES = [(np.cos(t), np.sin(t)) for t in (0.3, 1.1, 2.0, 2.9)]
# complex angles of the Sommerfeld integrals: k_rho on and off the real axis,
# below and beyond |k| (evanescent), k lossy
for k, kr in ((1.5 + 0.02j, 0.7), (1.5 + 0.02j, 2.6 - 0.4j), (2.0 + 0.01j, 1.9 - 0.3j), (1.0, 3.0 + 0.5j)):
    s = kr / k
    ANGLES.append((np.sqrt(1 - s * s), s))


@pytest.mark.parametrize("p", [4, 9, 12, 16])
def test_legendre_chebyshev_expansion(p):
    B = lmfmm.legendre_chebyshev(p)
    K = (p + 1) // 2
    assert B.shape == ((p + 1) * (p + 2) // 2, K + 1)
    for c, s in ANGLES:
        T = cheb(2 * c * c - 1, K)
        got = B @ T
        ref = f_ref(p, c, s)
        scale = np.maximum(np.abs(ref), np.abs(got)).max()
        assert np.max(np.abs(got - ref)) < 1e-12 * scale, (c, s)
        # the expansion is a polynomial in cos 2b: both branches of cos b agree
        np.testing.assert_allclose(f_ref(p, -c, -s), ref, rtol=1e-11, atol=1e-13 * scale)
    # entries beyond each function's degree in cos 2b are zero
    for n in range(p + 1):
        for m in range(n + 1):
            Kn = n // 2 if n % 2 == 0 else ((n + 1) // 2 if m % 2 == 0 else (n - 1) // 2)
            assert np.all(B[n * (n + 1) // 2 + m, Kn + 1:] == 0)


@pytest.mark.parametrize("p,k,kp", [(4, 1.0 + 0.02j, 1.5 + 0.02j), (8, 2.5 + 0.02j, 1.5 + 0.02j),
                                    (12, 0.8 + 0.01j, 2.0 + 0.01j), (12, 1.2, 1.2)])
def test_legendre_product_tensor(p, k, kp):
    G = lmfmm.legendre_product(p, k, kp)
    T = (p + 1) * (p + 2) // 2
    assert G.shape == (T, T, p + 2)
    k0 = k if abs(k) <= abs(kp) else kp
    for kr in (0.3, 1.1 + 0j, 2.2 - 0.35j, 3.1 + 0.2j):
        sb, sbp = kr / k, kr / kp
        cb, cbp = np.sqrt(1 - sb * sb), np.sqrt(1 - sbp * sbp)
        fs, ft = f_ref(p, cb, sb), f_ref(p, cbp, sbp)
        x0 = 1 - 2 * kr * kr / (k0 * k0)
        got = G @ cheb(x0, p + 1)
        ref = np.outer(fs, ft)
        scale = np.abs(ref).max()
        assert np.max(np.abs(got - ref)) < 1e-11 * scale, kr


def test_host_table_routines_reject_bad_arguments():
    with pytest.raises(lmfmm.LmfmmError):
        lmfmm.legendre_chebyshev(0)
    with pytest.raises(lmfmm.LmfmmError):
        lmfmm.legendre_product(17, 1.0, 1.0)
    with pytest.raises(lmfmm.LmfmmError):
        lmfmm.legendre_product(4, 0.0, 1.0)
