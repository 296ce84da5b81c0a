"""Pins for the CPU oracle: each check compares it with something other than
itself -- a library routine, a textbook closed form, a physical invariant, or
an independent route through the paper's formulas.  A plausible mistake in
the oracle (a dropped term, a wrong sign, a transposed slot, a wrong jump
condition) fails at least one of them.  All run on the CPU."""
import numpy as np
import pytest
import scipy.special as sp

import oracle as O
from paper_2507_18491_gb300 import workloads as W

D3 = [0.0, -1.2]
K3 = np.array([0.8, 1.5, 2.0]) + 0.01j
D4 = [0.0, -1.0, -2.0]
K4 = np.array([1.0, 1.5, 2.0, 2.5]) + 0.02j


def rel(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


# --------------------------------------------------------------- special fns
@pytest.mark.parametrize("z", [0.3, 7.3, 41.0, 380.5, 2.2 - 0.6j, -0.9j, 5.9 - 0.1j,
                               14.0 - 1.3j, 0.02 - 0.01j])
def test_besselj_matches_scipy(z):
    got = O.besselj(12, z)
    ref = sp.jv(np.arange(13), z)
    assert np.max(np.abs(got - ref)) < 5e-15 * max(1.0, np.max(np.abs(ref)))


def test_legendre_real_matches_scipy():
    th = 0.83
    P = O.legendre(9, np.cos(th), np.sin(th))
    for n in range(10):
        for m in range(n + 1):
            ref = sp.sph_harm_y(n, m, th, 0.0).real
            assert abs(P[n * (n + 1) // 2 + m] - ref) < 1e-14


def test_legendre_complex_closed_forms():
    # analytic extension with independent cos b, sin b (cos^2 + sin^2 = 1)
    k, kr = 1.3 + 0.02j, 2.7 - 0.4j
    kz = np.sqrt(k * k - kr * kr)
    kz = kz if kz.imag >= 0 else -kz
    c, s = kz / k, kr / k
    P = O.legendre(2, c, s)
    pi = np.pi
    ref = {(0, 0): 1 / np.sqrt(4 * pi), (1, 0): np.sqrt(3 / (4 * pi)) * c,
           (1, 1): -np.sqrt(3 / (8 * pi)) * s, (2, 0): np.sqrt(5 / (16 * pi)) * (3 * c * c - 1),
           (2, 1): -np.sqrt(15 / (8 * pi)) * s * c, (2, 2): np.sqrt(15 / (32 * pi)) * s * s}
    for (n, m), v in ref.items():
        assert abs(P[n * (n + 1) // 2 + m] - v) < 1e-14 * max(1, abs(v))


def test_plane_wave_expansion_complex_direction():
    """e^{iK.r} = 4 pi sum i^n j_n(kr) conj(Y_n^m(r^)) Y_n^m(K^) with the
    analytic extension cos b = k_z/k, sin b = k_rho/k (the ME/LE bases)."""
    k = 1.7 + 0.03j
    kr, alpha = 3.1 - 0.2j, 0.7
    kz = np.sqrt(k * k - kr * kr)
    kz = kz if kz.imag >= 0 else -kz
    r = np.array([0.11, -0.07, 0.09])
    K = np.array([kr * np.cos(alpha), kr * np.sin(alpha), kz])
    lhs = np.exp(1j * (K @ r))
    rn = np.linalg.norm(r)
    th, ph = np.arccos(r[2] / rn), np.arctan2(r[1], r[0])
    PK = O.legendre(30, kz / k, kr / k)
    tot = 0
    for n in range(31):
        jn = sp.spherical_jn(n, k * rn)
        for m in range(-n, n + 1):
            Yr = sp.sph_harm_y(n, m, th, ph)
            pk = PK[n * (n + 1) // 2 + abs(m)] * ((-1) ** m if m < 0 else 1)
            tot += 4 * np.pi * 1j ** n * jn * np.conj(Yr) * pk * np.exp(1j * m * alpha)
    assert abs(tot - lhs) < 1e-12 * abs(lhs)


# ------------------------------------------------------------- free space
@pytest.mark.parametrize("k", [1.3, 0.8 + 0.05j, 2.5])
@pytest.mark.parametrize("geom", [((0.3, -0.2, 0.9), (-0.1, 0.4, 0.2)),
                                  ((0.0, 0.0, 0.5), (0.0, 0.0, -0.4)),
                                  ((1.3, 0.8, 0.05), (-0.6, -0.4, 0.0))])
def test_free_space_spectral_equals_closed_form(k, geom):
    """Sommerfeld identity through the full J1..J5 assembly (eq. eq-GEGH-b-latest
    with phi^f, psi^f) against (I + grad grad/k^2) e^{ikR}/(4 pi R)."""
    r, rp = map(np.array, geom)
    assert rel(O.gfree_spectral(k, r, rp), O.gfree(k, r, rp)) < 1e-11


# ------------------------------------------------------------- 1-D problems
def test_homogeneous_stack():
    """Equal layers: same-layer reaction vanishes; a cross-layer pair carries
    the whole field (no free part is subtracted for l != l'), which must be the
    closed-form free-space dyadic; the only density is the direct one."""
    d = [0.0, -0.9]
    k = np.array([1.4, 1.4, 1.4]) + 0.01j
    for kr in [0.3, 1.2 - 0.3j, 5.0]:
        for l in range(3):
            for lp in range(3):
                ph, ps = O.densities(d, k, kr, l, lp)
                ref = np.zeros(4, complex)
                if l < lp:
                    ref[0] = 1.0       # up-up: e^{ik(z - z')}
                elif l > lp:
                    ref[3] = 1.0       # dn-dn: e^{ik(z' - z)}
                assert np.max(np.abs(ph - ref)) < 1e-13 and np.max(np.abs(ps - ref)) < 1e-13
    r, rs = np.array([0.2, 0.1, 0.4]), np.array([-0.3, 0.2, 0.7])
    assert np.max(np.abs(O.greact(d, k, r, rs))) < 1e-13
    rx = np.array([-0.3, 0.2, -1.5])
    assert rel(O.greact(d, k, r, rx), O.gfree(k[0], r, rx)) < 1e-10


def _kz(k, kr):
    s = np.sqrt(k * k - kr * kr + 0j)
    return s if s.imag >= 0 else -s


@pytest.mark.parametrize("kr", [0.4, 1.1 - 0.2j, 3.0])
def test_two_layer_fresnel(kr):
    """Half-space reflection/transmission: phi uses u' continuity (TE-like),
    psi uses (1/eps) u' continuity (TM-like), eps = k^2."""
    k = np.array([0.8, 1.2]) + 0.02j
    d = [0.0]
    k0, k1 = _kz(k[0], kr), _kz(k[1], kr)
    Y = {0: (k0, k1), 1: (k0 / k[0] ** 2, k1 / k[1] ** 2)}
    ph, ps = O.densities(d, k, kr, 0, 0)
    for dens, w in ((ph, 0), (ps, 1)):
        a, b = Y[w]
        assert abs(dens[1] - (a - b) / (a + b)) < 1e-14          # up-dn
        assert np.max(np.abs(dens[[0, 2, 3]])) == 0
    ph, ps = O.densities(d, k, kr, 1, 0)     # target below the source
    for dens, w in ((ph, 0), (ps, 1)):
        a, b = Y[w]
        assert abs(dens[3] - 2 * a / (a + b)) < 1e-14           # dn-dn
    ph, ps = O.densities(d, k, kr, 0, 1)     # target above the source
    for dens, w in ((ph, 0), (ps, 1)):
        a, b = Y[w]
        assert abs(dens[0] - 2 * b / (a + b)) < 1e-14           # up-up


@pytest.mark.parametrize("kr", [0.5, 1.7 - 0.25j, 4.0])
def test_slab_transmission_airy(kr):
    """Three layers, source above, target below: the textbook slab (Airy)
    transmission coefficient, times the Z-normalisation e^{-i k_2z T}."""
    T = 1.2
    d = [0.0, -T]
    k = np.array([0.8, 1.5, 2.0]) + 0.01j
    kz = [_kz(kk, kr) for kk in k]
    for w in (0, 1):
        Y = [kz[j] / (k[j] ** 2 if w else 1.0) for j in range(3)]
        r01 = (Y[0] - Y[1]) / (Y[0] + Y[1])
        r12 = (Y[1] - Y[2]) / (Y[1] + Y[2])
        t01 = 2 * Y[0] / (Y[0] + Y[1])
        t12 = 2 * Y[1] / (Y[1] + Y[2])
        e = np.exp(1j * kz[1] * T)
        tau = t01 * t12 * e / (1 + r01 * r12 * e * e)
        dens = O.densities(d, k, kr, 2, 0)[w]
        assert abs(dens[3] - tau * np.exp(-1j * kz[2] * T)) < 1e-13 * max(1, abs(tau))


def test_reaction_1d_interface_conditions():
    """u and (1/eta) du/dz continuous at every interface; the z'-derivative
    matches a central difference."""
    d, k = D4, K4
    kr = 1.3 - 0.2j
    for psi in (0, 1):
        for lp, zp in ((1, -0.4), (2, -1.7)):
            for i, di in enumerate(d):
                h = 1e-9
                a = O.reaction_1d(d, k, kr, psi, i, di + h, lp, zp)
                b = O.reaction_1d(d, k, kr, psi, i + 1, di - h, lp, zp)
                # add the free-space field of the source layer
                def free(l, z):
                    if l != lp:
                        return np.zeros(2, complex)
                    kz = _kz(k[lp], kr)
                    E = np.exp(1j * kz * abs(z - zp))
                    return np.array([-E / (2 * kz), -1j * np.sign(z - zp) * E / 2])
                ua = a[:2] + free(i, di + h)
                ub = b[:2] + free(i + 1, di - h)
                eta = (k[i] ** 2, k[i + 1] ** 2) if psi else (1.0, 1.0)
                assert abs(ua[0] - ub[0]) < 1e-8 * max(abs(ua[0]), 1e-3)
                assert abs(ua[1] / eta[0] - ub[1] / eta[1]) < 1e-8 * max(abs(ua[1] / eta[0]), 1e-3)
            hh = 1e-5
            c0 = O.reaction_1d(d, k, kr, psi, 0, 0.3, lp, zp)
            cp = O.reaction_1d(d, k, kr, psi, 0, 0.3, lp, zp + hh)
            cm = O.reaction_1d(d, k, kr, psi, 0, 0.3, lp, zp - hh)
            assert abs((cp[0] - cm[0]) / (2 * hh) - c0[2]) < 1e-8 * max(abs(c0[2]), 1e-3)
            assert abs((cp[1] - cm[1]) / (2 * hh) - c0[3]) < 1e-8 * max(abs(c0[3]), 1e-3)


# ------------------------------------------------------------ dyadic level
RNG = np.random.default_rng(7)


def _pts(d, layers, n):
    out = []
    d = np.asarray(d)
    for l in layers:
        top = d[l - 1] if l >= 1 else d[0] + 1.2
        bot = d[l] if l < d.size else d[-1] - 1.2
        for _ in range(n):
            out.append(np.array([RNG.uniform(-1, 1), RNG.uniform(-1, 1),
                                 RNG.uniform(bot + 0.05, top - 0.05)]))
    return out


@pytest.mark.parametrize("d,k", [(D3, K3), (D4, K4), ([0.0], np.array([0.8, 1.2]))])
def test_reciprocity(d, k):
    """G(r, r') = G(r', r)^T for mu = 1 (the symmetry the paper invokes to
    sum over the first slot)."""
    L = len(d)
    pts = _pts(d, range(L + 1), 2)
    for i in range(0, len(pts), 2):
        r, rp = pts[i], pts[(i + 3) % len(pts)]
        G1 = O.greact(d, k, r, rp)
        G2 = O.greact(d, k, rp, r)
        assert rel(G1, G2.T) < 1e-10


@pytest.mark.parametrize("d,k", [(D3, K3), (D4, K4)])
def test_sigma_route_equals_direct_route(d, k):
    """Eq. reactcompphysicaldomain (four components, densities sigma_1..5,
    image/effective maps, Z-exponentials, M-matrices) against the direct J1..J5
    assembly from the 1-D solution: two different routes through Section 3.1."""
    L = len(d)
    pts = _pts(d, range(L + 1), 2)
    for i in range(len(pts)):
        r, rp = pts[i], pts[(i * 5 + 3) % len(pts)]
        G1 = O.greact(d, k, r, rp)
        G2 = O.greact_sigma(d, k, r, rp)
        assert rel(G2, G1) < 1e-10


def test_printed_sigma3_differs_for_downward_targets():
    """The printed sigma_3 (sign tied to the source direction only) breaks the
    identity above for target-downward components; the reading
    sigma_3 = phi/k'_z + s_* s_star gamma k_z psi restores it."""
    r, rp = np.array([0.3, 0.2, -0.5]), np.array([-0.2, 0.1, -0.3])
    G1 = O.greact(D3, K3, r, rp)
    assert rel(O.greact_sigma(D3, K3, r, rp, literal=True), G1) > 1e-2
    assert rel(O.greact_sigma(D3, K3, r, rp, literal=False), G1) < 1e-10


def test_interface_continuity_of_total_field():
    """Tangential E continuous and eps E_z continuous across an interface for
    the total field (free part in the source layer + reaction)."""
    d, k = D3, K3
    rp = np.array([0.2, -0.1, 0.45])            # source in layer 0
    for di, (la, lb) in ((0.0, (0, 1)), (-1.2, (1, 2))):
        h = 1e-7
        ra = np.array([-0.3, 0.35, di + h])
        rb = np.array([-0.3, 0.35, di - h])
        Ga = O.greact(d, k, ra, rp, rtol=1e-13) + (O.gfree(k[0], ra, rp) if la == 0 else 0)
        Gb = O.greact(d, k, rb, rp, rtol=1e-13) + (O.gfree(k[0], rb, rp) if lb == 0 else 0)
        s = np.max(np.abs(Ga))
        assert np.max(np.abs(Ga[:2] - Gb[:2])) < 1e-5 * s
        assert np.max(np.abs(k[la] ** 2 * Ga[2] - k[lb] ** 2 * Gb[2])) < 1e-5 * s * abs(k[la]) ** 2


def test_direct_sum_is_sum_of_pairs():
    """or_direct sums G^r over the FIRST slot: Phi_i = sum_j G^r(r_j, r_i) q_j."""
    rng = np.random.default_rng(3)
    xyz = np.array(_pts(D3, [0, 1, 2], 3))
    J = rng.standard_normal((9, 3)) + 1j * rng.standard_normal((9, 3))
    phi, _ = O.direct(D3, K3, xyz, J, targets=[1, 5], rtol=1e-12)
    for t, i in enumerate([1, 5]):
        ref = sum(O.greact(D3, K3, xyz[j], xyz[i]) @ J[j] for j in range(9))
        assert rel(phi[t], ref) < 1e-10


def test_quadrature_tolerance_refinement():
    """Tightening the tolerance by 100x changes the result by less than the
    looser tolerance (the adaptive rule is converged, not merely stable)."""
    r, rp = np.array([0.9, -0.7, 0.12]), np.array([-0.8, 0.6, 0.15])
    G1 = O.greact([0.0], np.array([0.8, 1.2]), r, rp, rtol=1e-8)
    G2 = O.greact([0.0], np.array([0.8, 1.2]), r, rp, rtol=1e-12)
    assert rel(G1, G2) < 1e-8


def test_direct_free_is_the_sum_of_closed_form_dyads():
    """The oracle's free-space direct sum is sum_{j != i, same layer} of the
    closed-form dyad (itself pinned against the Sommerfeld assembly above)."""
    rng = np.random.default_rng(12)
    d, k = np.array([0.0, -1.2]), np.array([0.8, 1.5, 2.0]) + 0.01j
    xyz = W.points_in_layers(rng, d, [5, 4, 6], margin=0.1, xy=0.8)
    J = W.currents(rng, xyz.shape[0])
    got = O.direct_free(d, k, xyz, J)
    lay = [O.layer_of(d, z) for z in xyz[:, 2]]
    for i in range(xyz.shape[0]):
        ref = np.zeros(3, complex)
        for j in range(xyz.shape[0]):
            if j != i and lay[j] == lay[i]:
                ref += O.gfree(k[lay[i]], xyz[i], xyz[j]) @ J[j]
        np.testing.assert_allclose(got[i], ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())
