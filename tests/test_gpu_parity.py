"""GPU parity against the CPU oracle, stage by stage and end to end.

Tolerances: integer/index work is exact; floating point follows the FP64 bar
of a relative L2 error of 1e-6 for the FMM matvec (Err_2 of Section 4 over
the sampled targets), and tighter bars (1e-10 .. 1e-12) for stages that have
no truncation (densities, direct sums, tables)."""
import numpy as np
import pytest

import oracle as O
from paper_2507_18491_gb300 import lmfmm, workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

D2, K2 = np.array([0.0]), np.array([0.8, 1.2], dtype=complex)
D3, K3 = np.array([0.0, -1.2]), np.array([0.8, 1.5, 2.0]) + 0.01j
D4, K4 = np.array([0.0, -1.0, -2.0]), np.array([1.0, 1.5, 2.0, 2.5]) + 0.02j


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _ctx(d, k, p=4, xyz=None, **kw):
    prm = lmfmm.default_params()
    prm.p = p
    for a, v in kw.items():
        setattr(prm, a, v)
    ctx = lmfmm.create(prm, 0)
    lmfmm.set_layers(ctx, d, k)
    if xyz is not None:
        lmfmm.set_points(ctx, xyz)
    return ctx


# ------------------------------------------------------------------ a1
@pytest.mark.parametrize("d,k", [(D2, K2), (D3, K3), (D4, K4)])
def test_densities_match_oracle(d, k):
    ctx = _ctx(d, k)
    rng = np.random.default_rng(5)
    a = 1.5 * np.max(np.abs(k)) + 0.75
    kr = np.concatenate([rng.uniform(0.05, a, 6) - 1j * rng.uniform(0.05, 0.9, 6),
                         rng.uniform(a, 40.0, 6) + 0j, [0.3 + 0j, 2.0 - 0.5j]])
    L = d.size
    try:
        for l in range(L + 1):
            for lp in range(L + 1):
                kt = torch.from_numpy(kr.astype(np.complex128)).cuda()
                out = torch.empty((kr.size, 8), dtype=torch.complex128, device="cuda")
                lmfmm.densities(ctx, l, lp, kt, out)
                got = out.cpu().numpy()
                for q, x in enumerate(kr):
                    ph, ps = O.densities(d, k, x, l, lp)
                    ref = np.concatenate([ph, ps])
                    scale = max(np.max(np.abs(ref)), 1e-3)
                    assert np.max(np.abs(got[q] - ref)) < 1e-11 * scale, (l, lp, x)
    finally:
        lmfmm.destroy(ctx)


# ------------------------------------------------------------------ a6
@pytest.mark.parametrize("case", [
    (D2, K2, 0, 0, 1, 0, 0.0, 0.5, -0.5),
    (D2, K2, 0, 0, 1, 0, 0.9, 0.35, -0.6),
    (D3, K3, 1, 1, 0, 1, 1.3, -0.55, 0.9),    # same layer, down-up (s = -1)
    (D3, K3, 1, 1, 1, 0, 0.4, -0.3, -2.0),     # same layer, up-down
    (D3, K3, 0, 1, 1, 1, 0.7, 0.45, -0.5),     # target layer above
    (D3, K3, 2, 1, 0, 0, 1.1, -1.6, -0.6),     # target layer below (s = -1)
    (D4, K4, 2, 1, 1, 1, 0.6, -2.3, -1.4),
])
def test_m2l_tables_match_oracle(case):
    d, k, l, lp, tu, su, rho, zs, zt = case
    p = 4
    P = (p + 1) ** 2
    ctx = _ctx(d, k, p=p)
    try:
        out = torch.empty((5, P, P), dtype=torch.complex128, device="cuda")
        lmfmm.m2l_table(ctx, l, lp, tu, su, rho, zs, zt, out)
        got = out.cpu().numpy()
    finally:
        lmfmm.destroy(ctx)
    for t, (sig, kap) in enumerate(((1, 0), (5, 0), (2, 1), (4, 1), (3, 2))):
        ref = O.m2l_table(d, k, l, lp, tu, su, sig, kap, p, rho, zs, zt, rtol=1e-12).T
        # compare blockwise in (n', nu): entries span many orders of magnitude
        for n1 in range(p + 1):
            for nu in range(p + 1):
                rs = slice(nu * nu, (nu + 1) ** 2)
                cs = slice(n1 * n1, (n1 + 1) ** 2)
                r = ref[rs, cs]
                sc = np.max(np.abs(r))
                if sc == 0:
                    continue
                e = np.max(np.abs(got[t][rs, cs] - r)) / sc
                assert e < 1e-9, (t, n1, nu, e)


# ------------------------------------------------------------------ a10
def _pts3(rng, n_per):
    return W.points_in_layers(rng, D3, [n_per, n_per, n_per], margin=0.1, xy=0.8, height=1.0)


def test_direct_matches_oracle():
    rng = np.random.default_rng(21)
    xyz = _pts3(rng, 12)
    J = W.currents(rng, xyz.shape[0])
    ctx = _ctx(D3, K3, p=4, xyz=xyz, depth=1)
    try:
        lmfmm.build(ctx)
        Jt = torch.from_numpy(J).cuda()
        out = torch.empty_like(Jt)
        lmfmm.direct(ctx, Jt, out)
        got = out.cpu().numpy()
    finally:
        lmfmm.destroy(ctx)
    ref, _ = O.direct(D3, K3, xyz, J, rtol=1e-12)
    assert rel(got, ref) < 1e-8


# --------------------------------------------------------- full matvec
@pytest.mark.parametrize("p,theta,bar", [(6, 0.55, 1e-3), (10, 0.4, 1e-6)])
def test_matvec_two_layer_512_every_fourth_target(p, theta, bar):
    """The 512-point two-layer workload (depth 2) against the oracle computed
    now on every fourth target (every target is compared with the stored
    oracle sample in test_gpu_oracle_samples.py).  At its nominal p = 6 the
    truncation error is about 3e-4; p = 10 with theta = 0.4 meets the FP64
    bar of 1e-6."""
    w = W.two_layer_small()
    op = lmfmm.Operator(w.d, w.k, w.xyz, p=p, depth=w.depth, theta=theta).build()
    got = op.matvec(torch.from_numpy(w.J).cuda()).cpu().numpy()
    dref = op.direct(torch.from_numpy(w.J).cuda()).cpu().numpy()
    op.close()
    tg = np.arange(0, w.N, 4)
    ref, _ = O.direct(w.d, w.k, w.xyz, w.J, targets=tg)
    assert rel(dref[tg], ref) < 1e-8
    e = rel(got[tg], ref)
    assert e < bar, e


def test_matvec_three_layer_sparse_sources():
    """Config-2 medium at reduced N: all layers' components, deep tree; the
    oracle sums over a random subset of sources (J = 0 elsewhere)."""
    w = W.three_layer(n=8192, p=12, depth=4)
    rng = np.random.default_rng(3)
    src = rng.choice(w.N, 400, replace=False)
    J = np.zeros_like(w.J)
    J[src] = w.J[src]
    op = lmfmm.Operator(w.d, w.k, w.xyz, p=12, depth=4, theta=0.5).build()
    got = op.matvec(torch.from_numpy(J).cuda()).cpu().numpy()
    op.close()
    tg = rng.choice(w.N, 48, replace=False)
    ref, _ = O.direct(w.d, w.k, w.xyz, J, targets=tg, sources=src)
    assert rel(got[tg], ref) < 1e-6


def test_adjoint_identity():
    w = W.three_layer(n=2048, p=8, depth=3)
    op = lmfmm.Operator(w.d, w.k, w.xyz, p=8, depth=3).build()
    rng = np.random.default_rng(9)
    x = torch.from_numpy(W.currents(rng, w.N)).cuda()
    y = torch.from_numpy(W.currents(rng, w.N)).cuda()
    Ax = op.matvec(x)
    Ahy = op.rmatvec(y)
    lhs = torch.vdot(y.flatten(), Ax.flatten()).item()
    rhs = torch.vdot(Ahy.flatten(), x.flatten()).item()
    op.close()
    assert abs(lhs - rhs) < 1e-6 * abs(lhs)


def test_host_matvec_equals_device_matvec():
    w = W.two_layer_small(n=300, seed=4)
    op = lmfmm.Operator(w.d, w.k, w.xyz, p=6, depth=2).build()
    a = op.matvec(torch.from_numpy(w.J).cuda()).cpu().numpy()
    b = np.empty_like(w.J)
    lmfmm.matvec_host(op.ctx, np.ascontiguousarray(w.J), b)
    op.close()
    # the same operator; summation order of atomics may differ between calls
    assert rel(b, a) < 1e-13


def test_errors_are_reported_not_raised_on_device():
    prm = lmfmm.default_params()
    ctx = lmfmm.create(prm, 0)
    try:
        with pytest.raises(lmfmm.LmfmmError) as ei:
            lmfmm.set_points(ctx, np.zeros((3, 3)))
        assert ei.value.code == lmfmm.ERR_STATE
        lmfmm.set_layers(ctx, [0.0], [1.0, 2.0])
        with pytest.raises(lmfmm.LmfmmError) as ei:
            lmfmm.set_points(ctx, np.array([[0.0, 0.0, 0.0], [0.1, 0.2, 0.3]]))
        assert ei.value.code == lmfmm.ERR_ARG
        with pytest.raises(lmfmm.LmfmmError):
            lmfmm.set_layers(ctx, [0.0, 0.5], [1.0, 2.0, 1.5])
        with pytest.raises(lmfmm.LmfmmError):
            lmfmm.set_layers(ctx, [0.0], [1.0, 2.0 - 0.1j])
    finally:
        lmfmm.destroy(ctx)


def test_mixed_form_meets_its_bar():
    """FP32 translations (scaled expansions) against the oracle at 1e-5, and
    against the FP64 form of the same operator."""
    w = W.three_layer(n=8192, p=10, depth=4)
    rng = np.random.default_rng(4)
    src = rng.choice(w.N, 400, replace=False)
    J = np.zeros_like(w.J)
    J[src] = w.J[src]
    Jt = torch.from_numpy(J).cuda()
    op64 = lmfmm.Operator(w.d, w.k, w.xyz, p=10, depth=4, theta=0.5).build()
    a = op64.matvec(Jt).cpu().numpy()
    op64.close()
    op32 = lmfmm.Operator(w.d, w.k, w.xyz, p=10, depth=4, theta=0.5,
                          precision=lmfmm.MIXED).build()
    assert op32.stats()["m2l_kernel"] == 3      # default: persistent tensor-core M2L
    b = op32.matvec(Jt).cpu().numpy()
    op32.close()
    tg = rng.choice(w.N, 48, replace=False)
    ref, _ = O.direct(w.d, w.k, w.xyz, J, targets=tg, sources=src)
    assert rel(b[tg], ref) < 1e-5
    assert rel(b, a) < 2e-6


@pytest.mark.parametrize("p", [4, 7, 8, 12, 13, 15])
def test_tensor_core_m2l(p):
    """Mixed form with the M2L product on the tcgen05 tensor cores against the
    FP64 form, next to the FP32 SIMT product: the persistent kernel (three-piece
    bf16 split, p <= 12: 32 ... 176 table rows) and the streamed-operand kernel
    (three-term TF32 split, 1 to 4 row tiles of 128: 2P = 50 ... 512)."""
    w = W.three_layer(n=4096, p=p, depth=3)
    Jt = torch.from_numpy(w.J).cuda()
    kw = dict(p=p, depth=3, theta=0.5)
    op = lmfmm.Operator(w.d, w.k, w.xyz, **kw).build()
    a = op.matvec(Jt).cpu().numpy()
    op.close()
    out = {}
    expect = {0: 1, 1: 3 if p <= 12 else 2, 2: 2}
    for tc in (0, 1, 2):
        op = lmfmm.Operator(w.d, w.k, w.xyz, precision=lmfmm.MIXED, tensor_cores=tc, **kw).build()
        assert op.stats()["m2l_kernel"] == expect[tc]
        out[tc] = op.matvec(Jt).cpu().numpy()
        op.close()
    e = {tc: rel(out[tc], a) for tc in out}
    print("p=%d persistent %.3e  streamed %.3e  SIMT %.3e" % (p, e[1], e[2], e[0]))
    for tc in (1, 2):
        assert e[tc] < 5e-6 and e[tc] < 2 * e[0] + 1e-7


def test_tensor_core_translations():
    """tensor_cores = 3 also runs M2M / L2L on the persistent tensor-core kernel.
    Its truncating accumulation compounds along the tree; taking the inputs from
    the highest degree down keeps the added error small: within 1.5x the error of
    the M2L-only tensor-core form against the FP64 form, and close to that form."""
    w = W.three_layer(n=8192, p=12, depth=4)
    Jt = torch.from_numpy(w.J).cuda()
    kw = dict(p=12, depth=4, theta=0.5)
    op = lmfmm.Operator(w.d, w.k, w.xyz, **kw).build()
    a = op.matvec(Jt).cpu().numpy()
    op.close()
    out = {}
    for tc in (1, 3):
        op = lmfmm.Operator(w.d, w.k, w.xyz, precision=lmfmm.MIXED, tensor_cores=tc, **kw).build()
        assert op.stats()["m2l_kernel"] == 3
        out[tc] = op.matvec(Jt).cpu().numpy()
        op.close()
    print("M2L only %.3e  with translations %.3e" % (rel(out[1], a), rel(out[3], a)))
    assert rel(out[3], a) < 1.5 * rel(out[1], a) + 1e-7
    assert rel(out[3], out[1]) < 5e-6


def test_stats_before_first_matvec():
    w = W.two_layer_small(n=200, seed=5)
    op = lmfmm.Operator(w.d, w.k, w.xyz, p=6, depth=2).build()
    st = op.stats()
    assert st["n_points"] == 200 and st["ms_stage"]["total"] == 0
    op.matvec(torch.from_numpy(w.J).cuda())
    torch.cuda.synchronize()
    assert op.stats()["ms_stage"]["total"] > 0
    op.close()


def test_same_layer_tables_shared_by_equal_offsets():
    """The build keys same-layer tables on (level, rho, z_s - z_t): the device
    tabulation of two geometries with equal offsets gives the same table."""
    P = (8 + 1) ** 2
    ctx = _ctx(D4, K4, p=8)
    try:
        out = []
        for zs, zt in ((-0.2, -0.9), (-0.35, -1.05)):     # layer 1, images across z = 0
            t = torch.empty((5, P, P), dtype=torch.complex128, device="cuda")
            lmfmm.m2l_table(ctx, 1, 1, 1, 0, 0.35, zs + 0.6, zt, t)
            out.append(t.cpu().numpy())
    finally:
        lmfmm.destroy(ctx)
    for t in range(5):
        sc = np.max(np.abs(out[0][t]))
        assert np.max(np.abs(out[0][t] - out[1][t])) < 1e-13 * sc, t


def test_geometry_count_after_offset_merge():
    """Same-layer geometries of the four-layer clustered workload (N = 2^17,
    depth 4) are counted once per (level, rho, offset)."""
    w = W.four_layer_clusters(n=1 << 17)
    op = lmfmm.Operator(w.d, w.k, w.xyz, p=4, depth=4, theta=0.55).build()
    st = op.stats()
    op.close()
    assert 0 < st["n_geometries_same_layer"] < st["n_geometries"]
