"""CPU oracle for the layered-media Maxwell reaction field (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  It is a plain FP64 C implementation of the
definitions in Sections 3.1-3.5 of the paper (see ``lmfmm_oracle.c``) and
shares no code with the GPU library.

Parity pins (closed forms, invariants, brute force) live in
``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lmfmm_oracle.c")
_LIB = os.path.join(_HERE, "liblmfmm_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP).  Returns the library path."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp,
                               _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            D = ctypes.POINTER(ctypes.c_double)
            I64 = ctypes.POINTER(ctypes.c_int64)
            c_int, c_dbl = ctypes.c_int, ctypes.c_double
            lib.or_layer_of.argtypes = [c_int, D, c_dbl]
            lib.or_besselj.argtypes = [c_int, c_dbl, c_dbl, D]
            lib.or_reaction_1d.argtypes = [c_int, D, D, c_dbl, c_dbl, c_int, c_int, c_dbl,
                                           c_int, c_dbl, D]
            lib.or_densities.argtypes = [c_int, D, D, c_dbl, c_dbl, c_int, c_int, D]
            lib.or_sigmas.argtypes = [c_int, D, D, c_dbl, c_dbl, c_int, c_int, c_int, c_int,
                                      c_int, D]
            lib.or_greact.argtypes = [c_int, D, D, D, D, c_dbl, D]
            lib.or_greact.restype = c_int
            lib.or_greact_sigma.argtypes = [c_int, D, D, D, D, c_dbl, c_int, c_int, D]
            lib.or_greact_sigma.restype = c_int
            lib.or_gfree.argtypes = [c_dbl, c_dbl, D, D, D]
            lib.or_gfree_spectral.argtypes = [c_dbl, c_dbl, D, D, c_dbl, D]
            lib.or_direct.argtypes = [c_int, D, D, ctypes.c_int64, D, D, ctypes.c_int64, I64,
                                      ctypes.c_int64, I64, c_dbl, c_int, D]
            lib.or_direct.restype = ctypes.c_long
            lib.or_direct_free.argtypes = [c_int, D, D, ctypes.c_int64, D, D, ctypes.c_int64, I64,
                                           ctypes.c_int64, I64, c_int, D]
            lib.or_direct_free.restype = None
            lib.or_legendre.argtypes = [c_int, c_dbl, c_dbl, c_dbl, c_dbl, D]
            lib.or_m2l_table.argtypes = [c_int, D, D, c_int, c_int, c_int, c_int, c_int, c_int,
                                         c_int, c_int, c_dbl, c_dbl, c_dbl, c_dbl, D]
            lib.or_m2l_table.restype = c_int
            _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _medium(d, k):
    d = np.ascontiguousarray(np.asarray(d, float).reshape(-1))
    k = np.ascontiguousarray(np.asarray(k, complex).reshape(-1))
    assert k.size == d.size + 1
    kri = np.ascontiguousarray(np.stack([k.real, k.imag], 1).reshape(-1))
    return d.size, d, kri


def _c(a, n):
    return a.reshape(n, 2) @ np.array([1.0, 1j])


def layer_of(d, z):
    lib = _load()
    d = np.ascontiguousarray(np.asarray(d, float))
    return lib.or_layer_of(d.size, _dp(d), float(z))


def besselj(nmax, z):
    """J_0..J_nmax(z) (real z: C library jn; complex z: Bessel's integral)."""
    out = np.zeros(2 * (nmax + 1))
    _load().or_besselj(nmax, float(np.real(z)), float(np.imag(z)), _dp(out))
    return _c(out, nmax + 1)


def reaction_1d(d, k, krho, psi, l, z, lp, zp):
    """(u, du/dz, du/dz', d2u/dz dz') of the reaction part of phi (psi=0) or
    psi (psi=1) at z in layer l for the source at z' in layer lp."""
    L, d, kri = _medium(d, k)
    out = np.zeros(8)
    _load().or_reaction_1d(L, _dp(d), _dp(kri), float(np.real(krho)), float(np.imag(krho)),
                           int(psi), int(l), float(z), int(lp), float(zp), _dp(out))
    return _c(out, 4)


def densities(d, k, krho, l, lp):
    """phi^{*star}, psi^{*star} (order up-up, up-dn, dn-up, dn-dn)."""
    L, d, kri = _medium(d, k)
    out = np.zeros(16)
    _load().or_densities(L, _dp(d), _dp(kri), float(np.real(krho)), float(np.imag(krho)),
                         int(l), int(lp), _dp(out))
    v = _c(out, 8)
    return v[:4], v[4:]


def sigmas(d, k, krho, l, lp, tgt_up, src_up, literal=False):
    L, d, kri = _medium(d, k)
    out = np.zeros(10)
    _load().or_sigmas(L, _dp(d), _dp(kri), float(np.real(krho)), float(np.imag(krho)),
                      int(l), int(lp), int(tgt_up), int(src_up), int(literal), _dp(out))
    return _c(out, 5)


def greact(d, k, r, rp, rtol=1e-12):
    """Reaction part G^r(r, r') (3x3) of the electric dyadic Green's function."""
    L, d, kri = _medium(d, k)
    r = np.ascontiguousarray(r, float)
    rp = np.ascontiguousarray(rp, float)
    out = np.zeros(18)
    rc = _load().or_greact(L, _dp(d), _dp(kri), _dp(r), _dp(rp), float(rtol), _dp(out))
    if rc:
        raise ValueError("point on an interface")
    return _c(out, 9).reshape(3, 3)


def greact_sigma(d, k, r, rp, rtol=1e-12, literal=False, comps=(0, 1, 2, 3)):
    """G^r(r, r') through the four components and the densities sigma_1..5.

    ``comps`` selects components: 0 up-up, 1 up-dn, 2 dn-up, 3 dn-dn
    (target direction, source direction)."""
    mask = sum(1 << c for c in comps)
    L, d, kri = _medium(d, k)
    r = np.ascontiguousarray(r, float)
    rp = np.ascontiguousarray(rp, float)
    out = np.zeros(18)
    rc = _load().or_greact_sigma(L, _dp(d), _dp(kri), _dp(r), _dp(rp), float(rtol),
                                 int(literal), int(mask), _dp(out))
    if rc:
        raise ValueError("point on an interface")
    return _c(out, 9).reshape(3, 3)


def gfree(k, r, rp):
    out = np.zeros(18)
    r = np.ascontiguousarray(r, float)
    rp = np.ascontiguousarray(rp, float)
    _load().or_gfree(float(np.real(k)), float(np.imag(k)), _dp(r), _dp(rp), _dp(out))
    return _c(out, 9).reshape(3, 3)


def gfree_spectral(k, r, rp, rtol=1e-12):
    out = np.zeros(18)
    r = np.ascontiguousarray(r, float)
    rp = np.ascontiguousarray(rp, float)
    _load().or_gfree_spectral(float(np.real(k)), float(np.imag(k)), _dp(r), _dp(rp),
                              float(rtol), _dp(out))
    return _c(out, 9).reshape(3, 3)


def direct(d, k, xyz, J, targets=None, sources=None, rtol=1e-10, nthreads=0):
    """Phi_i = sum_j G^r(r_j, r_i) J_j for i in ``targets`` (all if None),
    j in ``sources`` (all if None).  Returns (Phi [nt,3] complex, calls)."""
    L, d, kri = _medium(d, k)
    xyz = np.ascontiguousarray(xyz, float)
    N = xyz.shape[0]
    q = np.ascontiguousarray(np.stack([J.real, J.imag], -1).reshape(-1))
    t = np.arange(N, dtype=np.int64) if targets is None else np.ascontiguousarray(targets,
                                                                                  np.int64)
    phi = np.zeros(6 * t.size)
    if sources is None:
        sp, ns = None, 0
    else:
        s = np.ascontiguousarray(sources, np.int64)
        sp, ns = s.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), s.size
    n = _load().or_direct(L, _dp(d), _dp(kri), N, _dp(xyz), _dp(q), t.size,
                          t.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), ns, sp,
                          float(rtol), int(nthreads), _dp(phi))
    return phi.reshape(-1, 3, 2) @ np.array([1.0, 1j]), n


def direct_free(d, k, xyz, J, targets=None, sources=None, nthreads=0):
    """Free-space part Phi^f_i = sum_{j != i, same layer} G_E^f(r_i, r_j) J_j
    (closed-form dyad) for i in ``targets`` (all if None), j in ``sources``."""
    L, d, kri = _medium(d, k)
    xyz = np.ascontiguousarray(xyz, float)
    N = xyz.shape[0]
    q = np.ascontiguousarray(np.stack([J.real, J.imag], -1).reshape(-1))
    t = np.arange(N, dtype=np.int64) if targets is None else np.ascontiguousarray(targets, np.int64)
    phi = np.zeros(6 * t.size)
    if sources is None:
        sp, ns = None, 0
    else:
        s = np.ascontiguousarray(sources, np.int64)
        sp, ns = s.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), s.size
    _load().or_direct_free(L, _dp(d), _dp(kri), N, _dp(xyz), _dp(q), t.size,
                           t.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), ns, sp, int(nthreads),
                           _dp(phi))
    return phi.reshape(-1, 3, 2) @ np.array([1.0, 1j])


def legendre(nmax, cosb, sinb):
    """Normalised P^_n^m(cos b), 0<=m<=n<=nmax, flat index n(n+1)/2+m."""
    cnt = (nmax + 1) * (nmax + 2) // 2
    out = np.zeros(2 * cnt)
    _load().or_legendre(nmax, float(np.real(cosb)), float(np.imag(cosb)),
                        float(np.real(sinb)), float(np.imag(sinb)), _dp(out))
    return _c(out, cnt)


def m2l_table(d, k, l, lp, tgt_up, src_up, sig, kappa, p, rho, zs, zt, rtol=1e-11,
              literal=False):
    """I-hat[(n',m'), (nu,mu)] (index n^2+n+m) for one (sigma, kappa)."""
    L, d, kri = _medium(d, k)
    P = (p + 1) ** 2
    out = np.zeros(2 * P * P)
    rc = _load().or_m2l_table(L, _dp(d), _dp(kri), int(l), int(lp), int(tgt_up), int(src_up),
                              int(literal), int(sig), int(kappa), int(p), float(rho),
                              float(zs), float(zt), float(rtol), _dp(out))
    if rc:
        raise ValueError("m2l_table: bad geometry (rc=%d)" % rc)
    return _c(out, P * P).reshape(P, P)
