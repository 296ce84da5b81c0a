"""Thin ctypes binding of the lmfmm C ABI (include/lmfmm.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Device buffers are torch tensors (complex128, contiguous); streams
are torch CUDA streams.  Importing this module does not build anything; if
the compiled library is missing it raises, so no silent fallback exists.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_lib = None

OK, ERR_ARG, ERR_CUDA, ERR_OOM, ERR_STATE, ERR_QUAD, ERR_UNSUPPORTED, ERR_TIMEOUT, ERR_INTERNAL = (
    0, -1, -2, -3, -4, -5, -6, -7, -8)
PLAN_DROP_FAR_PAIR, PLAN_DROP_NEAR_PAIR = 1, 2
FP64, MIXED = 0, 1
C128, C64 = 0, 1
REACTION, FREE, TOTAL = 0, 1, 2


class _Complex128(ctypes.Structure):
    _fields_ = [("re", ctypes.c_double), ("im", ctypes.c_double)]


class Params(ctypes.Structure):
    _fields_ = [("p", ctypes.c_int), ("depth", ctypes.c_int), ("leaf_cap", ctypes.c_int),
                ("theta", ctypes.c_double), ("eta", ctypes.c_double),
                ("quad_tol", ctypes.c_double), ("precision", ctypes.c_int),
                ("tensor_cores", ctypes.c_int), ("quad_node_cap", ctypes.c_int),
                ("components", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("n_points", ctypes.c_int64), ("n_layers", ctypes.c_int),
                ("n_components", ctypes.c_int), ("depth", ctypes.c_int),
                ("n_boxes", ctypes.c_int64), ("n_m2l_pairs", ctypes.c_int64),
                ("n_geometries", ctypes.c_int64), ("n_near_pairs", ctypes.c_int64),
                ("n_near_point_pairs", ctypes.c_int64), ("n_quad_nodes", ctypes.c_int64),
                ("bytes_tables", ctypes.c_double), ("ms_setup", ctypes.c_double),
                ("ms_stage", ctypes.c_double * 8), ("m2l_columns", ctypes.c_int64),
                ("m2l_kernel", ctypes.c_int), ("launches", ctypes.c_int),
                ("n_geometries_same_layer", ctypes.c_int64), ("ms_tabulate", ctypes.c_double),
                ("tab_flops", ctypes.c_double), ("adjoint_transposed", ctypes.c_int),
                ("n_free_geometries", ctypes.c_int64), ("n_free_near_point_pairs", ctypes.c_int64)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("depth", ctypes.c_int), ("n_components", ctypes.c_int),
                ("n_free_components", ctypes.c_int), ("n_components_unchecked", ctypes.c_int),
                ("n_boxes", ctypes.c_int64), ("n_leaves", ctypes.c_int64 * 9),
                ("n_far_pairs", ctypes.c_int64), ("n_geometries", ctypes.c_int64),
                ("n_near_pairs", ctypes.c_int64), ("n_near_point_pairs", ctypes.c_int64),
                ("n_free_far_pairs", ctypes.c_int64), ("n_free_geometries", ctypes.c_int64),
                ("n_free_near_pairs", ctypes.c_int64), ("n_free_near_point_pairs", ctypes.c_int64),
                ("n_translation_pairs", ctypes.c_int64), ("n_work_items", ctypes.c_int64),
                ("n_columns", ctypes.c_int64), ("n_leaf_pairs_checked", ctypes.c_int64),
                ("n_violations", ctypes.c_int64), ("root_center", ctypes.c_double * 3),
                ("root_half", ctypes.c_double), ("n_geometries_level", ctypes.c_int64 * 21),
                ("max_geometries_component_level", ctypes.c_int64), ("message", ctypes.c_char * 256)]


EXPORTS = ["lmfmm_default_params", "lmfmm_create", "lmfmm_set_layers", "lmfmm_set_points",
           "lmfmm_set_points_device", "lmfmm_build", "lmfmm_matvec", "lmfmm_matvec_host",
           "lmfmm_matvec_adjoint", "lmfmm_matvec_transpose", "lmfmm_gradient", "lmfmm_check", "lmfmm_test_set_status", "lmfmm_direct",
           "lmfmm_direct_noalloc", "lmfmm_densities", "lmfmm_m2l_table", "lmfmm_translation_matrix",
           "lmfmm_free_m2l_table", "lmfmm_legendre_chebyshev", "lmfmm_legendre_product",
           "lmfmm_get_stats", "lmfmm_plan_check", "lmfmm_plan_depth", "lmfmm_last_error", "lmfmm_destroy", "lmfmm_batch_create",
           "lmfmm_batch_matvec", "lmfmm_batch_tune", "lmfmm_batch_check", "lmfmm_batch_info",
           "lmfmm_batch_last_error", "lmfmm_batch_destroy"]


class LmfmmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("lmfmm error %d: %s" % (code, msg))
        self.code = code


def library_path() -> str:
    return _build.LIB


def load():
    """Load the compiled library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError("liblmfmm.so is not built (run paper_2507_18491_gb300.build.build())")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    i, i64, d = ctypes.c_int, ctypes.c_int64, ctypes.c_double
    sig = {
        "lmfmm_default_params": [ctypes.POINTER(Params)],
        "lmfmm_create": [ctypes.POINTER(P), ctypes.POINTER(Params), i],
        "lmfmm_set_layers": [P, i, ctypes.POINTER(d), ctypes.POINTER(_Complex128)],
        "lmfmm_set_points": [P, i64, ctypes.POINTER(d)],
        "lmfmm_set_points_device": [P, i64, P, P],
        "lmfmm_build": [P, P],
        "lmfmm_matvec": [P, P, i, P, P],
        "lmfmm_matvec_host": [P, P, i, P, P],
        "lmfmm_matvec_adjoint": [P, P, i, P, P],
        "lmfmm_matvec_transpose": [P, P, i, P, P],
        "lmfmm_gradient": [P, P, P, i, P, P, P],
        "lmfmm_check": [P, P],
        "lmfmm_test_set_status": [P, i],
        "lmfmm_direct": [P, P, P, P],
        "lmfmm_direct_noalloc": [P, P, P, P],
        "lmfmm_densities": [P, i, i, i64, P, P, P],
        "lmfmm_m2l_table": [P, i, i, i, i, d, d, d, P, P],
        "lmfmm_translation_matrix": [i, _Complex128, ctypes.POINTER(d), P, P],
        "lmfmm_free_m2l_table": [i, _Complex128, d, d, P, P],
        "lmfmm_get_stats": [P, ctypes.POINTER(Stats)],
        "lmfmm_legendre_chebyshev": [i, P],
        "lmfmm_legendre_product": [i, _Complex128, _Complex128, P],
        "lmfmm_plan_check": [ctypes.POINTER(Params), i, ctypes.POINTER(d), ctypes.POINTER(_Complex128), i64,
                             ctypes.POINTER(d), i, ctypes.POINTER(PlanInfo)],
        "lmfmm_plan_depth": [ctypes.POINTER(Params), i, ctypes.POINTER(d), ctypes.POINTER(_Complex128), i64,
                             ctypes.POINTER(d), i, i, ctypes.POINTER(d), ctypes.POINTER(i), ctypes.POINTER(d)],
        "lmfmm_last_error": [P],
        "lmfmm_destroy": [P],
        "lmfmm_batch_create": [ctypes.POINTER(P), ctypes.POINTER(P), i],
        "lmfmm_batch_matvec": [P, ctypes.POINTER(P), ctypes.POINTER(P), i, P],
        "lmfmm_batch_tune": [P, P],
        "lmfmm_batch_check": [P, P],
        "lmfmm_batch_info": [P, ctypes.POINTER(i), ctypes.POINTER(i64), ctypes.POINTER(i),
                             ctypes.POINTER(d)],
        "lmfmm_batch_last_error": [P],
        "lmfmm_batch_destroy": [P],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.lmfmm_last_error.restype = ctypes.c_char_p
    lib.lmfmm_destroy.restype = None
    lib.lmfmm_batch_last_error.restype = ctypes.c_char_p
    lib.lmfmm_batch_destroy.restype = None
    _lib = lib
    return lib


def _check(rc, ctx=None):
    if rc != OK:
        msg = load().lmfmm_last_error(ctx)
        raise LmfmmError(rc, msg.decode() if msg else "")


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _dptr(t, n3=None):
    import torch
    if not (t.is_cuda and t.dtype == torch.complex128 and t.is_contiguous()):
        raise ValueError("expected a contiguous complex128 CUDA tensor")
    if n3 is not None and tuple(t.shape) != (n3, 3):
        raise ValueError("expected shape (%d, 3), got %s" % (n3, tuple(t.shape)))
    return ctypes.c_void_p(t.data_ptr())


def _field(t, like=None):
    """(pointer, dtype code) of a contiguous complex128/complex64 CUDA tensor [N, 3]."""
    import torch
    codes = {torch.complex128: C128, torch.complex64: C64}
    if not (t.is_cuda and t.dtype in codes and t.is_contiguous() and t.dim() == 2
            and t.shape[1] == 3):
        raise ValueError("expected a contiguous complex128 or complex64 CUDA tensor [N, 3]")
    if like is not None and (t.dtype != like.dtype or t.shape != like.shape):
        raise ValueError("input and output must have the same dtype and shape")
    return ctypes.c_void_p(t.data_ptr()), codes[t.dtype]


# ------------------------------------------------------------ C-ABI mirror
def default_params() -> Params:
    prm = Params()
    _check(load().lmfmm_default_params(ctypes.byref(prm)))
    return prm


def create(prm: Params, device: int = 0):
    h = ctypes.c_void_p()
    _check(load().lmfmm_create(ctypes.byref(h), ctypes.byref(prm), int(device)))
    return h


def set_layers(ctx, d, k):
    d = np.ascontiguousarray(np.asarray(d, np.float64).reshape(-1))
    k = np.asarray(k, np.complex128).reshape(-1)
    karr = (_Complex128 * k.size)(*[_Complex128(float(v.real), float(v.imag)) for v in k])
    _check(load().lmfmm_set_layers(ctx, int(d.size), d.ctypes.data_as(ctypes.POINTER(
        ctypes.c_double)), karr), ctx)


def set_points(ctx, xyz):
    xyz = np.ascontiguousarray(np.asarray(xyz, np.float64).reshape(-1, 3))
    _check(load().lmfmm_set_points(ctx, int(xyz.shape[0]),
                                   xyz.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), ctx)


def set_points_device(ctx, xyz, stream=None):
    """Points from a contiguous float64 CUDA tensor [N, 3]."""
    import torch
    if not (xyz.is_cuda and xyz.dtype == torch.float64 and xyz.is_contiguous() and xyz.dim() == 2
            and xyz.shape[1] == 3):
        raise ValueError("expected a contiguous float64 CUDA tensor [N, 3]")
    _check(load().lmfmm_set_points_device(ctx, int(xyz.shape[0]), ctypes.c_void_p(xyz.data_ptr()),
                                          _stream(stream)), ctx)


def build(ctx, stream=None):
    _check(load().lmfmm_build(ctx, _stream(stream)), ctx)


def matvec(ctx, J, Phi, stream=None):
    """Phi = A J on the device (complex128 or complex64 tensors [N, 3], same dtype)."""
    pj, code = _field(J)
    pp, _ = _field(Phi, like=J)
    _check(load().lmfmm_matvec(ctx, pj, code, pp, _stream(stream)), ctx)


def matvec_adjoint(ctx, y, Phi, stream=None):
    py, code = _field(y)
    pp, _ = _field(Phi, like=y)
    _check(load().lmfmm_matvec_adjoint(ctx, py, code, pp, _stream(stream)), ctx)


def matvec_transpose(ctx, y, out, stream=None):
    py, code = _field(y)
    po, _ = _field(out, like=y)
    _check(load().lmfmm_matvec_transpose(ctx, py, code, po, _stream(stream)), ctx)


def gradient(ctx, J, g, gJ=None, gxyz=None, stream=None):
    """gJ = A^H g and gxyz = Re sum conj(g) dE/dr (FP64 form; see lmfmm_gradient)."""
    import torch
    pj, code = _field(J)
    pg, _ = _field(g, like=J)
    pgj = _field(gJ, like=J)[0] if gJ is not None else None
    if gxyz is not None and not (gxyz.is_cuda and gxyz.dtype == torch.float64 and gxyz.is_contiguous()
                                 and tuple(gxyz.shape) == (J.shape[0], 3)):
        raise ValueError("gxyz must be a contiguous float64 CUDA tensor [N, 3]")
    pgx = ctypes.c_void_p(gxyz.data_ptr()) if gxyz is not None else None
    _check(load().lmfmm_gradient(ctx, pj, pg, code, pgj, pgx, _stream(stream)), ctx)


def check(ctx, stream=None):
    """Wait for the stream and raise if a device wait of the matvecs gave up."""
    _check(load().lmfmm_check(ctx, _stream(stream)), ctx)


def test_set_status(ctx, bits):
    _check(load().lmfmm_test_set_status(ctx, int(bits)), ctx)


def matvec_host(ctx, J: np.ndarray, Phi: np.ndarray, stream=None):
    codes = {np.dtype(np.complex128): C128, np.dtype(np.complex64): C64}
    for a in (J, Phi):
        if a.dtype not in codes or not a.flags.c_contiguous:
            raise ValueError("expected contiguous complex128 or complex64 arrays")
    if J.dtype != Phi.dtype or J.shape != Phi.shape:
        raise ValueError("J and Phi must have the same dtype and shape")
    _check(load().lmfmm_matvec_host(ctx, ctypes.c_void_p(J.ctypes.data), codes[J.dtype],
                                    ctypes.c_void_p(Phi.ctypes.data), _stream(stream)), ctx)


def direct(ctx, J, Phi, stream=None):
    _check(load().lmfmm_direct(ctx, _dptr(J), _dptr(Phi), _stream(stream)), ctx)


def direct_noalloc(ctx, J, Phi, stream=None):
    """lmfmm_direct without device allocation (fixed 32 MiB device scratch)."""
    _check(load().lmfmm_direct_noalloc(ctx, _dptr(J), _dptr(Phi), _stream(stream)), ctx)


def densities(ctx, l, lp, krho, out, stream=None):
    _check(load().lmfmm_densities(ctx, int(l), int(lp), int(krho.numel()), _dptr(krho),
                                  _dptr(out), _stream(stream)), ctx)


def m2l_table(ctx, l, lp, tgt_up, src_up, rho, zs, zt, out, stream=None):
    _check(load().lmfmm_m2l_table(ctx, int(l), int(lp), int(tgt_up), int(src_up), float(rho),
                                  float(zs), float(zt), _dptr(out), _stream(stream)), ctx)


def translation_matrix(p, k, t):
    """(M2M, L2L) matrices [P, P] (numpy complex128) for wavenumber k and
    shift t = child centre - parent centre.  Host only."""
    P = (p + 1) ** 2
    up = np.zeros((P, P), np.complex128)
    dn = np.zeros((P, P), np.complex128)
    t = np.ascontiguousarray(np.asarray(t, np.float64))
    _check(load().lmfmm_translation_matrix(int(p), _Complex128(float(np.real(k)), float(np.imag(k))),
                                           t.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                           ctypes.c_void_p(up.ctypes.data),
                                           ctypes.c_void_p(dn.ctypes.data)))
    return up, dn


def free_m2l_table(p, k, rho, dz, blocks=False):
    """(tables [5, P, P], blocks [3, 3, P, P] or None) of the free-space M2L for
    c_s - c_t = (rho, 0, dz).  Host only."""
    P = (p + 1) ** 2
    tab = np.zeros((5, P, P), np.complex128)
    blk = np.zeros((3, 3, P, P), np.complex128) if blocks else None
    _check(load().lmfmm_free_m2l_table(int(p), _Complex128(float(np.real(k)), float(np.imag(k))),
                                       float(rho), float(dz), ctypes.c_void_p(tab.ctypes.data),
                                       ctypes.c_void_p(blk.ctypes.data) if blocks else None))
    return tab, blk


def legendre_chebyshev(p):
    """B[(p+1)(p+2)/2][(p+1)//2 + 1] of lmfmm_legendre_chebyshev (host only)."""
    B = np.zeros(((p + 1) * (p + 2) // 2, (p + 1) // 2 + 1))
    _check(load().lmfmm_legendre_chebyshev(int(p), ctypes.c_void_p(B.ctypes.data)))
    return B


def legendre_product(p, k, kp):
    """G[T][T][p+2] of lmfmm_legendre_product (host only)."""
    T = (p + 1) * (p + 2) // 2
    G = np.zeros((T, T, p + 2), np.complex128)
    _check(load().lmfmm_legendre_product(int(p), _Complex128(float(np.real(k)), float(np.imag(k))),
                                         _Complex128(float(np.real(kp)), float(np.imag(kp))),
                                         ctypes.c_void_p(G.ctypes.data)))
    return G


def get_stats(ctx) -> dict:
    s = Stats()
    _check(load().lmfmm_get_stats(ctx, ctypes.byref(s)), ctx)
    out = {f: getattr(s, f) for f, _ in Stats._fields_ if f != "ms_stage"}
    names = ["p2m", "m2m", "m2l", "l2l", "l2p", "s2t", "permute", "total"]
    out["ms_stage"] = {n: s.ms_stage[i] for i, n in enumerate(names)}
    return out


def plan_check(d, k, xyz, p=8, depth=-1, leaf_cap=64, theta=0.55, eta=0.1, components=REACTION, flags=0):
    """Host-only build and consistency check of the setup structures
    (lmfmm_plan_check); returns (status, info dict).  Needs no GPU."""
    prm = default_params()
    prm.p, prm.depth, prm.leaf_cap = int(p), int(depth), int(leaf_cap)
    prm.theta, prm.eta, prm.components = float(theta), float(eta), int(components)
    d = np.ascontiguousarray(np.asarray(d, np.float64).reshape(-1))
    k = np.asarray(k, np.complex128).reshape(-1)
    karr = (_Complex128 * k.size)(*[_Complex128(float(v.real), float(v.imag)) for v in k])
    xyz = np.ascontiguousarray(np.asarray(xyz, np.float64).reshape(-1, 3))
    info = PlanInfo()
    rc = load().lmfmm_plan_check(ctypes.byref(prm), int(d.size), d.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                 karr, int(xyz.shape[0]), xyz.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                 int(flags), ctypes.byref(info))
    out = {f: getattr(info, f) for f, _ in PlanInfo._fields_
           if f not in ("n_leaves", "root_center", "message", "n_geometries_level")}
    out["n_leaves"] = list(info.n_leaves)[:d.size + 1]
    out["n_geometries_level"] = list(info.n_geometries_level)[:info.depth + 1]
    out["root_center"] = list(info.root_center)
    out["message"] = info.message.decode()
    return rc, out


def plan_depth(d, k, xyz, p=8, depths=(4, 5, 6, 7), theta=0.55, eta=0.1, components=REACTION, unit_ns=None):
    """Leaf-level tuner (lmfmm_plan_depth, host only): returns (best depth,
    {depth: predicted matvec ms})."""
    prm = default_params()
    prm.p, prm.theta, prm.eta, prm.components = int(p), float(theta), float(eta), int(components)
    d = np.ascontiguousarray(np.asarray(d, np.float64).reshape(-1))
    k = np.asarray(k, np.complex128).reshape(-1)
    karr = (_Complex128 * k.size)(*[_Complex128(float(v.real), float(v.imag)) for v in k])
    xyz = np.ascontiguousarray(np.asarray(xyz, np.float64).reshape(-1, 3))
    d0, d1 = int(min(depths)), int(max(depths))
    pred = (ctypes.c_double * (d1 - d0 + 1))()
    best = ctypes.c_int()
    u = None
    if unit_ns is not None:
        u = (ctypes.c_double * 4)(*[float(x) for x in unit_ns])
    _check(load().lmfmm_plan_depth(ctypes.byref(prm), int(d.size), d.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                   karr, int(xyz.shape[0]), xyz.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                   d0, d1, u, ctypes.byref(best), pred))
    return best.value, {d0 + j: pred[j] for j in range(d1 - d0 + 1)}


def last_error(ctx=None) -> str:
    m = load().lmfmm_last_error(ctx)
    return m.decode() if m else ""


def destroy(ctx):
    if ctx:
        load().lmfmm_destroy(ctx)


# ------------------------------------------------------------- convenience
class Operator:
    """The reaction-field operator of one point set in one layered medium.

    ``Operator(d, k, xyz, p=...)`` sets up the context; ``build()`` runs the
    setup on the GPU; ``matvec(J)`` returns A J (torch complex128 or complex64,
    [N,3], the dtype of J); ``check()`` raises if a device wait gave up."""

    def __init__(self, d, k, xyz, p=8, depth=-1, leaf_cap=64, theta=0.55, eta=0.1,
                 precision=FP64, tensor_cores=True, device=0, quad_node_cap=None,
                 components=REACTION):
        prm = default_params()
        prm.components = int(components)
        if quad_node_cap is not None:
            prm.quad_node_cap = int(quad_node_cap)
        prm.p, prm.depth, prm.leaf_cap = int(p), int(depth), int(leaf_cap)
        prm.theta, prm.eta, prm.precision = float(theta), float(eta), int(precision)
        prm.tensor_cores = int(tensor_cores)
        self.ctx = create(prm, device)
        self.N = int(np.asarray(xyz).shape[0])
        self.device = device
        set_layers(self.ctx, d, k)
        set_points(self.ctx, xyz)

    def build(self, stream=None):
        build(self.ctx, stream)
        return self

    def matvec(self, J, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty_like(J)
        matvec(self.ctx, J, out, stream)
        return out

    def rmatvec(self, y, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty_like(y)
        matvec_adjoint(self.ctx, y, out, stream)
        return out

    def tmatvec(self, y, out=None, stream=None):
        """A^T y with the transposed operators (FP64 / SIMT mixed forms)."""
        import torch
        if out is None:
            out = torch.empty_like(y)
        matvec_transpose(self.ctx, y, out, stream)
        return out

    def vjp(self, J, g, stream=None):
        """(A^H g, Re sum conj(g) dE/dr) for E = A(r) J (FP64 form)."""
        import torch
        gJ = torch.empty_like(J)
        gx = torch.empty((J.shape[0], 3), dtype=torch.float64, device=J.device)
        gradient(self.ctx, J, g, gJ, gx, stream)
        return gJ, gx

    def check(self, stream=None):
        check(self.ctx, stream)

    def direct(self, J, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty_like(J)
        direct(self.ctx, J, out, stream)
        return out

    def stats(self):
        return get_stats(self.ctx)

    def close(self):
        if self.ctx:
            destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class ReactionField:
    """E = A(r) J as a differentiable torch function of the currents J and the
    point coordinates r (FP64 form).  ``ReactionField(d, k, xyz, **kw)`` builds
    the operator at the coordinates xyz; ``apply(J, xyz_tensor)`` returns E and,
    under autograd, backpropagates into J (A^H g) and into the coordinates
    (Re sum conj(g) dE/dr, tree and lists held fixed) through lmfmm_gradient,
    which recomputes the forward expansions it needs (checkpointed on the
    device) instead of keeping them from the forward call."""

    def __init__(self, d, k, xyz, **kw):
        kw.setdefault("precision", FP64)
        self.op = Operator(d, k, xyz, **kw).build()

    def apply(self, J, xyz):
        return _ReactionFieldFn.apply(J, xyz, self.op)

    def close(self):
        self.op.close()


def _make_fn():
    import torch

    class Fn(torch.autograd.Function):
        @staticmethod
        def forward(ctx, J, xyz, op):
            ctx.op = op
            ctx.save_for_backward(J)
            return op.matvec(J.contiguous())

        @staticmethod
        def backward(ctx, g):
            (J,) = ctx.saved_tensors
            gJ, gx = ctx.op.vjp(J.contiguous(), g.contiguous())
            return gJ, gx, None

    return Fn


class _LazyFn:
    _fn = None

    @classmethod
    def apply(cls, *args):
        if cls._fn is None:
            cls._fn = _make_fn()
        return cls._fn.apply(*args)


_ReactionFieldFn = _LazyFn


class Batch:
    """Several built Operators applied together (lmfmm_batch_*): one CUDA graph
    per set of buffers, the M2L of all problems in one persistent launch."""

    def __init__(self, ops):
        self.ops = list(ops)
        arr = (ctypes.c_void_p * len(self.ops))(*[o.ctx.value for o in self.ops])
        h = ctypes.c_void_p()
        rc = load().lmfmm_batch_create(ctypes.byref(h), arr, len(self.ops))
        if rc != OK:
            raise LmfmmError(rc, load().lmfmm_batch_last_error(None).decode())
        self.h = h

    def _check(self, rc):
        if rc != OK:
            raise LmfmmError(rc, load().lmfmm_batch_last_error(self.h).decode())

    def matvec(self, Js, outs, stream=None):
        n = len(self.ops)
        codes = [_field(J)[1] for J in Js]
        for J, o in zip(Js, outs):
            _field(o, like=J)
        if len(set(codes)) != 1 or len(Js) != n or len(outs) != n:
            raise ValueError("one J and one output per problem, all of one dtype")
        pj = (ctypes.c_void_p * n)(*[J.data_ptr() for J in Js])
        po = (ctypes.c_void_p * n)(*[o.data_ptr() for o in outs])
        self._keep = (pj, po)
        self._check(load().lmfmm_batch_matvec(self.h, pj, po, codes[0], _stream(stream)))
        return outs

    def tune(self, stream=None):
        self._check(load().lmfmm_batch_tune(self.h, _stream(stream)))

    def check(self, stream=None):
        self._check(load().lmfmm_batch_check(self.h, _stream(stream)))

    def info(self):
        m, v = ctypes.c_int(), ctypes.c_int()
        nw = ctypes.c_int64()
        ms = (ctypes.c_double * 4)()
        self._check(load().lmfmm_batch_info(self.h, ctypes.byref(m), ctypes.byref(nw), ctypes.byref(v), ms))
        return {"merged": bool(m.value), "nwork": nw.value, "variant": v.value, "ms_variant": list(ms)}

    def close(self):
        if getattr(self, "h", None):
            load().lmfmm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
