"""M2M / L2L matrices of the regular expansions (host code, no GPU), pinned
by closed forms: a single source at the child centre has the one-term ME
sqrt(4 pi) delta_{n0}; its exact ME about the parent centre is
4 pi j_n(k|t|) conj(Y_n^m(t^)).  Likewise the LE L_00 = 1 (the field
j_0(k|x|) Y_0^0) re-expands about a child centre as
sqrt(4 pi) (-1)^n j_n(k|t|) conj(Y_n^m(t^)) (Gegenbauer's addition theorem).
These fix every entry of column 0 to relative precision.  The full matrices
are checked against an independent sphere quadrature of
int e^{ik K.t} Y_n'm' conj(Y_nm) dOmega (absolute accuracy)."""
import numpy as np
import pytest
import scipy.special as sp

from paper_2507_18491_gb300 import build, lmfmm


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()


def _closed(p, k, t, sign):
    tn = np.linalg.norm(t)
    th, ph = np.arccos(t[2] / tn), np.arctan2(t[1], t[0])
    out = np.zeros((p + 1) ** 2, complex)
    for n in range(p + 1):
        jn = sp.spherical_jn(n, k * tn)
        for m in range(-n, n + 1):
            out[n * n + n + m] = np.sqrt(4 * np.pi) * (sign ** n) * jn * np.conj(
                sp.sph_harm_y(n, m, th, ph))
    return out


@pytest.mark.parametrize("p,k,t", [(8, 1.3, (0.1, -0.2, 0.15)),
                                   (12, 2.5 + 0.02j, (-0.03, 0.03, -0.03)),
                                   (12, 0.8 + 0.01j, (0.4, 0.4, -0.4))])
def test_column0_closed_forms(p, k, t):
    up, dn = lmfmm.translation_matrix(p, k, t)
    t = np.array(t)
    for col, ref in ((up[:, 0], _closed(p, k, t, 1)), (dn[:, 0], _closed(p, k, t, -1))):
        # relative to each degree block (entries shrink like (k|t|)^n/(2n+1)!!)
        for n in range(p + 1):
            b = slice(n * n, (n + 1) ** 2)
            assert np.max(np.abs(col[b] - ref[b])) < 1e-12 * np.max(np.abs(ref[b])), n


def test_full_matrix_against_sphere_quadrature():
    p, k, t = 6, 1.7 + 0.03j, np.array([0.25, -0.1, 0.3])
    up, dn = lmfmm.translation_matrix(p, k, t)
    nth, nph = 40, 80
    x, wx = np.polynomial.legendre.leggauss(nth)
    th = np.arccos(x)
    ph = 2 * np.pi * np.arange(nph) / nph
    TH, PH = np.meshgrid(th, ph, indexing="ij")
    W = (wx[:, None] * np.ones(nph)[None, :] * 2 * np.pi / nph).ravel()
    K = np.stack([np.sin(TH) * np.cos(PH), np.sin(TH) * np.sin(PH), np.cos(TH)], -1).reshape(-1, 3)
    E = np.exp(1j * k * (K @ t))
    P = (p + 1) ** 2
    Y = np.zeros((K.shape[0], P), complex)
    for n in range(p + 1):
        for m in range(-n, n + 1):
            Y[:, n * n + n + m] = sp.sph_harm_y(n, m, TH.ravel(), PH.ravel())
    Wm = (np.conj(Y) * (W * E)[:, None]).T @ Y
    nn = np.array([int(np.sqrt(i)) for i in range(P)])
    ref_up = (1j ** (nn[None, :] - nn[:, None])) * Wm
    ref_dn = (1j ** (nn[:, None] - nn[None, :])) * Wm
    assert np.max(np.abs(up - ref_up)) < 1e-13
    assert np.max(np.abs(dn - ref_dn)) < 1e-13


def test_zero_shift_is_identity():
    up, dn = lmfmm.translation_matrix(10, 1.1, (0.0, 0.0, 0.0))
    assert np.max(np.abs(up - np.eye(121))) < 1e-14
    assert np.max(np.abs(dn - np.eye(121))) < 1e-14
