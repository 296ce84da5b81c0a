"""Gradient of a least-squares objective of the field, f = sum_i |E_i - E_ref,i|^2
with E = A(r) J (FP64 form): with respect to J it is A^H g (g = 2 (E - E_ref)),
with respect to the coordinates Re sum conj(g) dE/dr (lmfmm_gradient, through
torch.autograd as well).  Checked against central finite differences (h = 1e-6)
of the FMM itself, rebuilt at the displaced points, and against finite
differences of the oracle's direct sum on a small case."""
import numpy as np
import pytest

import oracle as O
from paper_2507_18491_gb300 import lmfmm, workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _f(w, xyz, J, Eref, kw):
    op = lmfmm.Operator(w.d, w.k, xyz, **kw).build()
    try:
        E = op.matvec(J).cpu().numpy()
    finally:
        op.close()
    return float(np.sum(np.abs(E - Eref) ** 2))


def _setup(n, p, depth, seed=5):
    w = W.three_layer(n=n, p=p, depth=depth, seed=1002)
    rng = np.random.default_rng(seed)
    Jref = W.currents(rng, w.N)
    kw = dict(p=p, depth=depth, theta=0.5)
    op = lmfmm.Operator(w.d, w.k, w.xyz, **kw).build()
    Eref = op.matvec(torch.from_numpy(Jref).cuda()).cpu().numpy()
    J = torch.from_numpy(w.J).cuda()
    E = op.matvec(J)
    g = 2.0 * (E - torch.from_numpy(Eref).cuda())
    gJ, gx = op.vjp(J, g)
    adj = op.rmatvec(g)
    st = op.stats()
    op.close()
    return w, J, Eref, kw, gJ.cpu().numpy(), gx.cpu().numpy(), adj.cpu().numpy(), st


def test_gradient_against_finite_differences_of_the_fmm():
    w, J, Eref, kw, gJ, gx, adj, st = _setup(800, 8, 2)
    assert st["n_near_point_pairs"] > 0
    np.testing.assert_allclose(gJ, adj, rtol=0, atol=1e-12 * np.abs(adj).max())
    h = 1e-6
    rng = np.random.default_rng(1)
    pts = rng.choice(w.N, 6, replace=False)
    worst = 0.0
    scale = np.abs(gx).max()
    for j in pts:
        for a in range(3):
            xp, xm = w.xyz.copy(), w.xyz.copy()
            xp[j, a] += h
            xm[j, a] -= h
            fd = (_f(w, xp, J, Eref, kw) - _f(w, xm, J, Eref, kw)) / (2 * h)
            worst = max(worst, abs(fd - gx[j, a]) / scale)
    print("coordinate gradient vs central differences: worst %.3e of max |grad| %.3e" % (worst, scale))
    assert worst < 1e-5


def test_gradient_directional_derivative_three_layer_32768():
    """The adjoint configuration's size: N = 32768, p = 10; 32 random
    coordinates displaced at once along a random direction (h = 1e-6; the
    tree, lists and quadrature rules are those of the undisplaced points)."""
    w, J, Eref, kw, gJ, gx, adj, st = _setup(32768, 10, 4)
    rng = np.random.default_rng(3)
    v = np.zeros(w.xyz.shape)
    idx = rng.choice(w.xyz.size, 32, replace=False)
    v.flat[idx] = rng.standard_normal(32)
    h = 1e-6
    fd = (_f(w, w.xyz + h * v, J, Eref, kw) - _f(w, w.xyz - h * v, J, Eref, kw)) / (2 * h)
    an = float(np.sum(gx * v))
    print("directional derivative: analytic %.9e  central differences %.9e" % (an, fd))
    assert abs(an - fd) < 1e-6 * abs(an)


def test_autograd_function_matches_vjp():
    w = W.three_layer(n=500, p=6, depth=2)
    rf = lmfmm.ReactionField(w.d, w.k, w.xyz, p=6, depth=2)
    try:
        J = torch.from_numpy(w.J).cuda().requires_grad_(True)
        x = torch.from_numpy(w.xyz).cuda().requires_grad_(True)
        E = rf.apply(J, x)
        loss = torch.sum(torch.abs(E) ** 2)
        loss.backward()
        gJ, gx = rf.op.vjp(J.detach(), 2.0 * E.detach())
    finally:
        rf.close()
    assert torch.allclose(J.grad, gJ, rtol=0, atol=1e-12 * gJ.abs().max().item())
    assert torch.allclose(x.grad, gx, rtol=0, atol=1e-12 * gx.abs().max().item())


def test_gradient_against_the_oracle():
    """Finite differences of the oracle's direct sum (the exact operator) at a
    few coordinates of a small three-layer case, against the FMM's analytic
    gradient at high order."""
    rng = np.random.default_rng(8)
    d, k = np.array([0.0, -1.2]), np.array([0.8, 1.5, 2.0]) + 0.01j
    xyz = W.points_in_layers(rng, d, [30, 30, 30], margin=0.1, xy=0.8)
    J = W.currents(rng, xyz.shape[0])
    Eref = W.currents(rng, xyz.shape[0])
    op = lmfmm.Operator(d, k, xyz, p=14, depth=1, theta=0.4).build()
    try:
        Jt = torch.from_numpy(J).cuda()
        E = op.matvec(Jt)
        g = 2.0 * (E - torch.from_numpy(Eref).cuda())
        _, gx = op.vjp(Jt, g)
        gx = gx.cpu().numpy()
    finally:
        op.close()

    def f_oracle(x):
        Eo, _ = O.direct(d, k, x, J, rtol=1e-12)
        return float(np.sum(np.abs(Eo - Eref) ** 2))

    h = 1e-5
    worst = 0.0
    for j, a in ((3, 0), (40, 2), (75, 1), (12, 2)):
        xp, xm = xyz.copy(), xyz.copy()
        xp[j, a] += h
        xm[j, a] -= h
        fd = (f_oracle(xp) - f_oracle(xm)) / (2 * h)
        worst = max(worst, abs(fd - gx[j, a]) / np.abs(gx).max())
    print("FMM gradient vs oracle differences: worst %.3e" % worst)
    assert worst < 1e-5
