"""ctypes wrappers of the plain-C FP64 oracle (hisq_oracle.c).

Test infrastructure; see oracle/__init__.py.  Arrays are NumPy complex128,
C-contiguous: links [4][V][3][3], spinor blocks [N][V/2][3].
"""
from __future__ import annotations

import ctypes as ct

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ct.CDLL(path)
        P = ct.c_void_p
        I = ct.c_int
        D = ct.c_double
        L.oracle_dslash.argtypes = [P, P, P, I, P, P, I, I]
        L.oracle_apply_A.argtypes = [P, P, P, I, D, P, P, I]
        L.oracle_apply_A_sites.argtypes = [P, P, P, I, D, P, P, ct.c_long, P]
        L.oracle_cg.argtypes = [P, P, P, I, D, P, P, I, D, I, P, P]
        L.oracle_cg_iterates.argtypes = [P, P, P, I, D, P, P, I]
        L.oracle_link_grad.argtypes = [P, P, P, I, P, P, I, P, P]
        L.oracle_set_threads.argtypes = [I]
        for f in (L.oracle_dslash, L.oracle_apply_A, L.oracle_apply_A_sites, L.oracle_cg,
                  L.oracle_cg_iterates, L.oracle_link_grad, L.oracle_set_threads):
            f.restype = I
        _lib = L
    return _lib


def _c(a, dtype=np.complex128):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a


def _dims(dims):
    return np.ascontiguousarray(np.asarray(dims, dtype=np.int32))


def _p(a):
    return a.ctypes.data_as(ct.c_void_p)


def _check_links(dims, fat, lng):
    V = int(np.prod(dims))
    fat = _c(fat)
    lng = _c(lng)
    assert fat.shape == (4, V, 3, 3) and lng.shape == (4, V, 3, 3)
    return fat, lng


def dslash(dims, fat, lng, psi, out_parity: int, antiperiodic_t: bool = False) -> np.ndarray:
    """D restricted to out_parity <- 1-out_parity, on a block [N][V/2][3] (Eq. 2)."""
    fat, lng = _check_links(dims, fat, lng)
    psi = _c(psi)
    squeeze = psi.ndim == 2
    if squeeze:
        psi = psi[None]
    out = np.empty_like(psi)
    d = _dims(dims)
    rc = lib().oracle_dslash(_p(d), _p(fat), _p(lng), int(antiperiodic_t), _p(psi), _p(out),
                             int(out_parity), psi.shape[0])
    assert rc == 0, rc
    return out[0] if squeeze else out


def apply_A(dims, fat, lng, mass: float, v, antiperiodic_t: bool = False) -> np.ndarray:
    """A v = m^2 v - D_eo D_oe v on even sites (Sec. 3.2)."""
    fat, lng = _check_links(dims, fat, lng)
    v = _c(v)
    squeeze = v.ndim == 2
    if squeeze:
        v = v[None]
    out = np.empty_like(v)
    d = _dims(dims)
    rc = lib().oracle_apply_A(_p(d), _p(fat), _p(lng), int(antiperiodic_t), float(mass), _p(v),
                              _p(out), v.shape[0])
    assert rc == 0, rc
    return out[0] if squeeze else out


def apply_A_sites(dims, fat, lng, mass: float, v, sites, antiperiodic_t: bool = False):
    """(A v)(x) at the given even lexicographic sites; v is one column [V/2][3]."""
    fat, lng = _check_links(dims, fat, lng)
    v = _c(v)
    assert v.ndim == 2
    sites = np.ascontiguousarray(np.asarray(sites, dtype=np.int64))
    out = np.empty((len(sites), 3), dtype=np.complex128)
    d = _dims(dims)
    rc = lib().oracle_apply_A_sites(_p(d), _p(fat), _p(lng), int(antiperiodic_t), float(mass),
                                    _p(v), _p(sites), len(sites), _p(out))
    assert rc == 0, rc
    return out


def cg(dims, fat, lng, mass: float, b, tol: float, max_iter: int = 100000, x0=None,
       antiperiodic_t: bool = False):
    """N independent textbook CG solves of A x_j = b_j.  Returns (x, iters, true_rel_res)."""
    fat, lng = _check_links(dims, fat, lng)
    b = _c(b)
    if b.ndim == 2:
        b = b[None]
    x = np.zeros_like(b) if x0 is None else _c(x0).copy()
    n = b.shape[0]
    iters = np.zeros(n, dtype=np.int32)
    res = np.zeros(n, dtype=np.float64)
    d = _dims(dims)
    rc = lib().oracle_cg(_p(d), _p(fat), _p(lng), int(antiperiodic_t), float(mass), _p(b), _p(x),
                         n, float(tol), int(max_iter), _p(iters), _p(res))
    assert rc in (0, 1), rc
    return x, iters, res


def cg_iterates(dims, fat, lng, mass: float, b, n_iter: int, antiperiodic_t: bool = False):
    """x after exactly n_iter plain CG iterations from x0 = 0 (one column)."""
    fat, lng = _check_links(dims, fat, lng)
    b = _c(b)
    assert b.ndim == 2
    x = np.empty_like(b)
    d = _dims(dims)
    rc = lib().oracle_cg_iterates(_p(d), _p(fat), _p(lng), int(antiperiodic_t), float(mass),
                                  _p(b), _p(x), int(n_iter))
    assert rc == 0, rc
    return x


def link_grad(dims, fat, lng, x, lam, antiperiodic_t: bool = False):
    """Gradient (dL/dRe + i dL/dIm) of a real loss with respect to the fat and
    long links, given x = A^-1 phi and the adjoint lam = A^-1 dL/dx (even-site
    blocks [N][V/2][3]); returns (gfat, glong), each [4][V][3][3]."""
    fat, lng = _check_links(dims, fat, lng)
    x = _c(x)
    lam = _c(lam)
    if x.ndim == 2:
        x, lam = x[None], lam[None]
    assert x.shape == lam.shape
    gf = np.empty_like(fat)
    gl = np.empty_like(lng)
    d = _dims(dims)
    rc = lib().oracle_link_grad(_p(d), _p(fat), _p(lng), int(antiperiodic_t), _p(x), _p(lam),
                                x.shape[0], _p(gf), _p(gl))
    assert rc == 0, rc
    return gf, gl


def set_threads(n: int) -> int:
    """OpenMP threads of the oracle's loops; returns the previous setting."""
    return lib().oracle_set_threads(int(n))
