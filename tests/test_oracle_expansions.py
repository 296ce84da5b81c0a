"""Pin of the far-field chain of Section 3.3 (eqs. mecoeff, metoleimage1,
M2L_scale_with_Tnmu, maxwell_LE_layered) for single reaction components:
a source point's multipole expansion (ME) about its image-side centre,
translated by the M2L built from the oracle's Sommerfeld integrals I-hat, and
evaluated as a local expansion (LE) at the target's effective location, must
converge in p to the component dyad G^{*star}(r_j, r_i) computed directly.

The M2L coefficient used here, derived from the plane-wave expansions of
Section 3.3 with eq. general_integral_I_Alternative, is
  T[nu mu, n' m'] = (-i)^nu i^(n'+1+d) s^(nu+mu+n'+m') e^{i d phi} I-hat,
  d = m' - mu + kappa,
and the 3x3 tensor of eq. Tnm_nmu_M2L acts, in helical components
(a, b, c) = (q_x + i q_y, q_x - i q_y, q_z), as
  A' = 1/2 T0[s1] a - 1/2 T2[s3] b + T1[s2] c
  B' = 1/2 T0[s1] b - 1/2 T-2[s3] a + T-1[s2] c
  C' = T0[s5] c + 1/2 T-1[s4] a + 1/2 T1[s4] b.
The GPU library implements exactly this chain, so this test is the bridge
between the paper's formulas and the kernels."""
import numpy as np
import pytest
import scipy.special as sp

import oracle as O

D3 = np.array([0.0, -1.2])
K3 = np.array([0.8, 1.5, 2.0]) + 0.01j


def _tau_hat(d, l, lp, tu, su, z):
    if tu and su:
        return z if l < lp else 2 * d[l] - z
    if tu and not su:
        return z if l <= lp else 2 * d[l] - z
    if not tu and su:
        return 2 * d[l - 1] - z if l < lp else z
    return 2 * d[l - 1] - z if l <= lp else z


def _tau_breve(d, l, lp, su, z):
    if not su:
        return 2 * d[lp] - z if l <= lp else z
    return z if l < lp else 2 * d[lp - 1] - z


def _s(l, lp, su):
    return (1 if l < lp else -1) if su else (1 if l <= lp else -1)


def _sph(v):
    r = np.linalg.norm(v)
    return r, np.arccos(np.clip(v[2] / r, -1, 1)), np.arctan2(v[1], v[0])


def _chain(d, k, l, lp, tu, su, rj, ri, q, cs_off, ct_off, p):
    kk, kp = k[l], k[lp]
    s = _s(l, lp, su)
    rb = np.array([rj[0], rj[1], _tau_hat(d, l, lp, tu, su, rj[2])])
    rbp = np.array([ri[0], ri[1], _tau_breve(d, l, lp, su, ri[2])])
    cs, ct = rb + cs_off, rbp + ct_off
    P = (p + 1) ** 2
    h = np.array([q[0] + 1j * q[1], q[0] - 1j * q[1], q[2]])
    rr, th, ph = _sph(rb - cs)
    M = np.zeros((3, P), complex)
    for n in range(p + 1):
        jn = sp.spherical_jn(n, kk * rr)
        for m in range(-n, n + 1):
            M[:, n * n + n + m] = 4 * np.pi * h * jn * np.conj(sp.sph_harm_y(n, m, th, ph))
    dx, dy = cs[0] - ct[0], cs[1] - ct[1]
    rho, phi = np.hypot(dx, dy), np.arctan2(dy, dx)
    T = {}
    for sig, kap in ((1, 0), (5, 0), (2, 1), (2, -1), (4, 1), (4, -1), (3, 2), (3, -2)):
        Ih = O.m2l_table(d, k, l, lp, tu, su, sig, kap, p, rho, cs[2], ct[2], rtol=1e-12)
        Tm = np.zeros((P, P), complex)
        for n1 in range(p + 1):
            for m1 in range(-n1, n1 + 1):
                for nu in range(p + 1):
                    for mu in range(-nu, nu + 1):
                        dd = m1 - mu + kap
                        c = (-1j) ** nu * 1j ** (n1 + 1 + dd) * s ** (nu + mu + n1 + m1)
                        Tm[nu * nu + nu + mu, n1 * n1 + n1 + m1] = (
                            c * np.exp(1j * dd * phi) * Ih[n1 * n1 + n1 + m1, nu * nu + nu + mu])
        T[(sig, kap)] = Tm
    a, b, c = M
    A = 0.5 * T[1, 0] @ a - 0.5 * T[3, 2] @ b + T[2, 1] @ c
    B = 0.5 * T[1, 0] @ b - 0.5 * T[3, -2] @ a + T[2, -1] @ c
    C = T[5, 0] @ c + 0.5 * T[4, -1] @ a + 0.5 * T[4, 1] @ b
    rr, th, ph = _sph(rbp - ct)
    basis = np.zeros(P, complex)
    for nu in range(p + 1):
        jn = sp.spherical_jn(nu, kp * rr)
        for mu in range(-nu, nu + 1):
            basis[nu * nu + nu + mu] = jn * sp.sph_harm_y(nu, mu, th, ph)
    Ah, Bh, Ch = A @ basis, B @ basis, C @ basis
    return np.array([(Ah + Bh) / 2, (Ah - Bh) / 2j, Ch])


@pytest.mark.parametrize("comp", [(0, 0, 1, 0), (1, 1, 0, 1), (1, 1, 1, 0), (1, 1, 0, 0),
                                  (1, 1, 1, 1), (0, 1, 1, 1), (1, 0, 0, 0), (2, 1, 0, 0),
                                  (0, 2, 1, 1)])
def test_me_m2l_le_chain_converges(comp):
    l, lp, tu, su = comp
    rng = np.random.default_rng(11 + 7 * l + 3 * lp + tu + 2 * su)

    def pt(layer):
        top = D3[layer - 1] if layer >= 1 else 1.2
        bot = D3[layer] if layer < 2 else -2.4
        return np.array([rng.uniform(-0.5, 0.5), rng.uniform(-0.5, 0.5),
                         rng.uniform(bot + 0.3, top - 0.3)])

    rj, ri = pt(l), pt(lp)
    q = rng.standard_normal(3) + 1j * rng.standard_normal(3)
    cs_off = np.array([0.02, -0.015, 0.025]) * (1 if rng.random() < 0.5 else -1)
    ct_off = np.array([-0.025, 0.01, 0.015]) * (1 if rng.random() < 0.5 else -1)
    ref = O.greact_sigma(D3, K3, rj, ri, rtol=1e-13, comps=[(0 if tu else 2) + (0 if su else 1)]) @ q
    errs = []
    for p in (3, 6):
        got = _chain(D3, K3, l, lp, tu, su, rj, ri, q, cs_off, ct_off, p)
        errs.append(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    assert errs[1] < 1e-6 and errs[1] < 0.05 * errs[0], errs


def test_same_layer_tables_depend_on_the_vertical_offset_only():
    """Eq. onedimensionintegral: within one layer (k = k') the vertical factor
    e^{i s (k_z z_s - k'_z z_t)} depends on z_s - z_t alone, so two M2L
    geometries of equal (rho, z_s - z_t) share a table; between layers they do
    not.  This is what lets the build key same-layer tables on the offset."""
    d, k = np.array([0.0, -1.2]), np.array([0.8, 1.5, 2.0]) + 0.01j
    p, rho = 3, 0.4
    # layer 1, target up / source down (s = +1): mapped source above the target
    a = O.m2l_table(d, k, 1, 1, 1, 0, 1, 0, p, rho, 0.30, -0.50, rtol=1e-13)
    b = O.m2l_table(d, k, 1, 1, 1, 0, 1, 0, p, rho, 0.45, -0.35, rtol=1e-13)
    assert np.max(np.abs(a - b)) < 1e-11 * np.max(np.abs(a))
    # layers 0 and 1 (k != k'): shifting both heights changes the table
    c = O.m2l_table(d, k, 0, 1, 1, 1, 1, 0, p, rho, 0.45, -0.5, rtol=1e-13)
    e = O.m2l_table(d, k, 0, 1, 1, 1, 1, 0, p, rho, 0.60, -0.35, rtol=1e-13)
    assert np.max(np.abs(c - e)) > 1e-3 * np.max(np.abs(c))


def test_table_entries_do_not_depend_on_the_truncation():
    """Each entry I-hat[(nu, mu), (n', m')] of eq. onedimensionintegral is its own
    Sommerfeld integral: the entries of degrees <= 2 computed in a p = 2 table
    and in a p = 9 table must agree entry by entry, although the p = 9 table
    also holds entries larger by many orders (the high-degree Legendre products
    grow like k_rho^(n + n')).  A tolerance shared by all entries of a table
    fails this for the small low-degree entries."""
    d, k = np.array([0.0, -1.0, -2.0]), np.array([1.0, 1.5, 2.0, 2.5]) + 0.02j
    # transmission from layer 2 up into layer 1, horizontal offset = vertical distance
    args = (d, k, 2, 1, 1, 1, 5, 0)
    small = O.m2l_table(*args, 2, 0.45, -1.2, -0.75, rtol=1e-12)
    big = O.m2l_table(*args, 9, 0.45, -1.2, -0.75, rtol=1e-12)[:9, :9]
    assert np.max(np.abs(big) / np.max(np.abs(small))) < 1e3
    rel = np.abs(big - small) / np.abs(small)
    assert np.max(rel) < 1e-10, np.max(rel)
