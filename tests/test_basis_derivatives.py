"""The derivative identities of the regular solid harmonics R_n^m = j_n(k r)
Y_n^m(r^) (orthonormal, Condon-Shortley) that the position-gradient kernels use
(CPU, against central differences of scipy's j_n and Y_n^m at complex k):
  d/dz R_n^m = k (a- R_{n-1}^m - a+ R_{n+1}^m)
  (d/dx + i d/dy) R_n^m = k (b+ R_{n+1}^{m+1} + b- R_{n-1}^{m+1})
  (d/dx - i d/dy) R_n^m = -k (c+ R_{n+1}^{m-1} + c- R_{n-1}^{m-1})."""
import numpy as np
import pytest

special = pytest.importorskip("scipy.special")

K = 1.3 + 0.2j


def R(n, m, r):
    if n < 0 or abs(m) > n:
        return 0.0
    x, y, z = r
    rr = np.sqrt(x * x + y * y + z * z)
    return special.spherical_jn(n, K * rr) * special.sph_harm_y(n, m, np.arccos(z / rr), np.arctan2(y, x))


def coef(n, m):
    s = lambda v: np.sqrt(max(v, 0.0))
    ap = s(((n + 1) ** 2 - m * m) / ((2 * n + 1) * (2 * n + 3)))
    am = s((n * n - m * m) / ((2 * n - 1) * (2 * n + 1))) if n > 0 else 0.0
    bp = s((n + m + 1) * (n + m + 2) / ((2 * n + 1) * (2 * n + 3)))
    bm = s((n - m) * (n - m - 1) / ((2 * n - 1) * (2 * n + 1))) if n > 0 else 0.0
    cp = s((n - m + 1) * (n - m + 2) / ((2 * n + 1) * (2 * n + 3)))
    cm = s((n + m) * (n + m - 1) / ((2 * n - 1) * (2 * n + 1))) if n > 0 else 0.0
    return ap, am, bp, bm, cp, cm


@pytest.mark.parametrize("r0", [(0.31, -0.22, 0.17), (-0.2, 0.4, -0.3), (0.05, 0.02, 0.6)])
def test_solid_harmonic_gradients(r0):
    r0 = np.array(r0)
    h = 1e-6
    for n in range(0, 7):
        for m in range(-n, n + 1):
            d = [(R(n, m, r0 + h * e) - R(n, m, r0 - h * e)) / (2 * h) for e in np.eye(3)]
            ap, am, bp, bm, cp, cm = coef(n, m)
            dz = K * (am * R(n - 1, m, r0) - ap * R(n + 1, m, r0))
            dp = K * (bp * R(n + 1, m + 1, r0) + bm * R(n - 1, m + 1, r0))
            dm = -K * (cp * R(n + 1, m - 1, r0) + cm * R(n - 1, m - 1, r0))
            assert abs(dz - d[2]) < 1e-8, (n, m)
            assert abs(dp - (d[0] + 1j * d[1])) < 1e-8, (n, m)
            assert abs(dm - (d[0] - 1j * d[1])) < 1e-8, (n, m)
