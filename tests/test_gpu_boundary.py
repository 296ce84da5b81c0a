"""The C-ABI boundary on the GPU: complex64 and complex128 caller buffers, the
device-pointer point upload, the status word of the asynchronous matvec (error
injected from the host, no device fault), and the quadrature node cap of the
build on its host-checked and device-flagged paths."""
import numpy as np
import pytest

from paper_2507_18491_gb300 import lmfmm, workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("precision", [lmfmm.FP64, lmfmm.MIXED])
def test_complex64_io_matches_complex128(precision):
    """complex64 currents are widened exactly, so A J agrees with the complex128
    call on the same (complex64-representable) currents up to the final
    rounding of Phi to complex64."""
    w = W.three_layer(n=4096, p=8, depth=3)
    J64 = torch.from_numpy(w.J.astype(np.complex64)).cuda()
    J128 = J64.to(torch.complex128)
    op = lmfmm.Operator(w.d, w.k, w.xyz, p=8, depth=3, precision=precision,
                        tensor_cores=3).build()
    try:
        a = op.matvec(J128).cpu().numpy()
        b = op.matvec(J64)
        assert b.dtype == torch.complex64
        b = b.cpu().numpy().astype(np.complex128)
        op.check()
        # host-buffer entry point with complex64 arrays
        Jh = np.ascontiguousarray(w.J.astype(np.complex64))
        Ph = np.empty_like(Jh)
        lmfmm.matvec_host(op.ctx, Jh, Ph)
    finally:
        op.close()
    # complex64 rounding of the result (2^-24) plus the atomics' summation order
    assert rel(b, a) < 2e-7
    assert rel(Ph.astype(np.complex128), a) < 2e-7


def test_mismatched_dtypes_are_rejected():
    w = W.two_layer_small(n=200, seed=5)
    op = lmfmm.Operator(w.d, w.k, w.xyz, p=4, depth=1).build()
    try:
        J = torch.from_numpy(w.J).cuda()
        with pytest.raises(ValueError):
            op.matvec(J, out=torch.empty(J.shape, dtype=torch.complex64, device="cuda"))
        rc = lmfmm.load().lmfmm_matvec(op.ctx, J.data_ptr(), 7, J.data_ptr(), None)
        assert rc == lmfmm.ERR_ARG
    finally:
        op.close()


def test_status_word_reaches_the_caller():
    """A wait that gives up inside a tensor-core kernel ORs bit 4 into the
    context's status word; lmfmm_check reports it after the stream is done, and
    the next matvec starts from a clear word.  The failure is injected from the
    host (no kernel is made to fail)."""
    w = W.three_layer(n=2048, p=6, depth=3)
    op = lmfmm.Operator(w.d, w.k, w.xyz, p=6, depth=3, precision=lmfmm.MIXED,
                        tensor_cores=3).build()
    try:
        J = torch.from_numpy(w.J).cuda()
        op.matvec(J)
        op.check()
        lmfmm.test_set_status(op.ctx, 4)
        with pytest.raises(lmfmm.LmfmmError) as ei:
            op.check()
        assert ei.value.code == lmfmm.ERR_TIMEOUT and "gave up" in str(ei.value)
        # the host-buffer entry point checks the word itself
        lmfmm.test_set_status(op.ctx, 4)
        op.matvec(J)          # clears the word before its first kernel
        op.check()
        Jh = np.ascontiguousarray(w.J)
        Ph = np.empty_like(Jh)
        lmfmm.matvec_host(op.ctx, Jh, Ph)
    finally:
        op.close()


def test_quad_node_cap_on_the_host_checked_tables():
    """An M2L table whose k_rho rule needs more nodes than quad_node_cap stops
    the build before any tabulation kernel runs."""
    w = W.three_layer(n=2048, p=6, depth=3)
    op = lmfmm.Operator(w.d, w.k, w.xyz, p=6, depth=3, quad_node_cap=64)
    try:
        with pytest.raises(lmfmm.LmfmmError) as ei:
            op.build()
        assert ei.value.code == lmfmm.ERR_QUAD and "quad_node_cap" in str(ei.value)
    finally:
        op.close()


def test_quad_node_cap_on_the_device_flagged_near_field():
    """With depth 0 every box pair is near: the near-field kernel meets the cap,
    clamps its rule (bounded work), sets the flag, and the build reports it."""
    w = W.three_layer(n=256, p=4, depth=0)
    op = lmfmm.Operator(w.d, w.k, w.xyz, p=4, depth=0, quad_node_cap=64)
    try:
        with pytest.raises(lmfmm.LmfmmError) as ei:
            op.build()
        assert ei.value.code == lmfmm.ERR_QUAD
    finally:
        op.close()
    # the same context builds with the default cap
    op = lmfmm.Operator(w.d, w.k, w.xyz, p=4, depth=0).build()
    op.close()


def test_set_points_device_equals_host_upload():
    w = W.three_layer(n=3000, p=6, depth=3)
    J = torch.from_numpy(w.J).cuda()
    op = lmfmm.Operator(w.d, w.k, w.xyz, p=6, depth=3).build()
    a = op.matvec(J).cpu().numpy()
    op.close()
    prm = lmfmm.default_params()
    prm.p, prm.depth = 6, 3
    ctx = lmfmm.create(prm, 0)
    try:
        lmfmm.set_layers(ctx, w.d, w.k)
        lmfmm.set_points_device(ctx, torch.from_numpy(w.xyz).cuda())
        lmfmm.build(ctx)
        out = torch.empty_like(J)
        lmfmm.matvec(ctx, J, out)
        b = out.cpu().numpy()
    finally:
        lmfmm.destroy(ctx)
    assert rel(b, a) < 1e-13
