"""The free-space M2L (Section 2: eq. maxwell_M2L_freespace, with the Hessian
of eq. GEandGH folded in) as the library builds it on the host, checked on the
CPU against the closed-form dyad G_E^f = (I + grad grad / k^2) e^{ikR}/(4 pi R):
a point source's multipole expansion (P2M of eq. mecoeff, written out with
scipy) is translated by the nine helical blocks, and by the five stored tables
with the M2L kernels' per-pair factors at a rotated azimuth, then evaluated as
a local expansion (eq. maxwell_LE_layered) at a target."""
import numpy as np
import pytest

import oracle as O
from paper_2507_18491_gb300 import build, lmfmm

special = pytest.importorskip("scipy.special")

K = 1.3 + 0.05j
P_ORDER = 14


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()
    lmfmm.load()


def sph(r):
    x, y, z = r
    rr = np.sqrt(x * x + y * y + z * z)
    return rr, np.arccos(z / rr), np.arctan2(y, x)


def nm_list(p):
    return [(n, m) for n in range(p + 1) for m in range(-n, n + 1)]


def p2m(rsrc, q, p):
    """Helical multipole expansions (a, b, c) of a point source at rsrc (box centre 0)."""
    rr, th, ph = sph(rsrc)
    qh = np.array([q[0] + 1j * q[1], q[0] - 1j * q[1], q[2]])
    b = np.array([4 * np.pi * special.spherical_jn(n, K * rr) * np.conj(special.sph_harm_y(n, m, th, ph))
                  for n, m in nm_list(p)])
    return qh[:, None] * b[None, :]


def l2p(L, r, p):
    rr, th, ph = sph(r)
    b = np.array([special.spherical_jn(n, K * rr) * special.sph_harm_y(n, m, th, ph) for n, m in nm_list(p)])
    A, B, C = L @ b
    return np.array([(A + B) / 2, (A - B) / 2j, C])


def kernel_apply(tab, phi, Mh, p):
    """The M2L kernels' use of the five tables for one pair at azimuth phi of
    c_s - c_t (s = +1, no mirrored boxes)."""
    idx = {nm: i for i, nm in enumerate(nm_list(p))}
    cols = [[(0, 0, 0.5, 0), (1, 0, 0.5, 1)], [(2, 0, 1.0, 2)], [(2, 1, 1.0, 0), (2, -1, 1.0, 1)],
            [(1, 1, 0.5, 2), (0, -1, 0.5, 2)], [(1, 2, -0.5, 0), (0, -2, -0.5, 1)]]
    L = np.zeros_like(Mh)
    for t in range(5):
        for vin, kap, cf, vout in cols[t]:
            x = np.zeros(len(idx), complex)
            for (n, m), k in idx.items():
                ms = -m if kap < 0 else m
                x[k] = 1j ** ((n + ms) % 4) * np.exp(1j * ms * phi) * Mh[vin, idx[(n, ms)]]
            y = tab[t] @ x
            c = cf * (-1.0 if kap < 0 and kap % 2 else 1.0)
            for (nu, mh), r in idx.items():
                mu = -mh if kap < 0 else mh
                L[vout, idx[(nu, mu)]] += c * (1j ** ((1 + kap) % 4)) * (1j ** ((-(nu + mu)) % 4)) \
                    * np.exp(1j * (kap - mu) * phi) * y[r]
    return L


@pytest.mark.parametrize("rho,dz", [(1.6, 0.7), (0.0, -1.8), (1.2, 0.0)])
def test_free_m2l_blocks_reproduce_the_free_dyad(rho, dz):
    p = P_ORDER
    tab, blk = lmfmm.free_m2l_table(p, K, rho, dz, blocks=True)
    cs, ct = np.array([0.0, 0.0, 0.0]), np.array([-rho, 0.0, -dz])    # c_s - c_t = (rho, 0, dz)
    rng = np.random.default_rng(4)
    for _ in range(3):
        rs = cs + 0.08 * rng.standard_normal(3)
        rt = ct + 0.08 * rng.standard_normal(3)
        q = rng.standard_normal(3) + 1j * rng.standard_normal(3)
        Mh = p2m(rs - cs, q, p)
        L = np.einsum("ovrc,vc->or", blk, Mh)
        got = l2p(L, rt - ct, p)
        ref = O.gfree(K, rt, rs) @ q
        assert np.linalg.norm(got - ref) < 1e-8 * np.linalg.norm(ref)


def test_free_m2l_tables_with_the_kernel_factors_at_any_azimuth():
    """The five tables with the per-pair factors e^{i m phi} (and the kappa < 0
    order flips) reproduce the dyad for a rotated box pair."""
    p = 12
    rho, dz, phi = 1.4, 0.9, 2.1
    tab, _ = lmfmm.free_m2l_table(p, K, rho, dz)
    cs = np.zeros(3)
    ct = cs - np.array([rho * np.cos(phi), rho * np.sin(phi), dz])
    rng = np.random.default_rng(6)
    for _ in range(3):
        rs = cs + 0.06 * rng.standard_normal(3)
        rt = ct + 0.06 * rng.standard_normal(3)
        q = rng.standard_normal(3) + 1j * rng.standard_normal(3)
        L = kernel_apply(tab, phi, p2m(rs - cs, q, p), p)
        got = l2p(L, rt - ct, p)
        ref = O.gfree(K, rt, rs) @ q
        assert np.linalg.norm(got - ref) < 1e-7 * np.linalg.norm(ref)
