"""Dense matrix of A = m^2 - D_eo D_oe on tiny lattices (2^4, 4^4).

Test infrastructure; see oracle/__init__.py.  Column k of the matrix is A
applied (by the C oracle) to the k-th unit vector of the even-site space, in
the (L,) = [V/2][3] flattening.
"""
from __future__ import annotations

import numpy as np

from . import hisq


def dense_A(dims, fat, lng, mass: float, antiperiodic_t: bool = False) -> np.ndarray:
    vh = int(np.prod(dims)) // 2
    L = 3 * vh
    units = np.eye(L, dtype=np.complex128).reshape(L, vh, 3)
    cols = hisq.apply_A(dims, fat, lng, mass, units, antiperiodic_t)
    return np.ascontiguousarray(cols.reshape(L, L).T)


def dense_D(dims, fat, lng, out_parity: int, antiperiodic_t: bool = False) -> np.ndarray:
    vh = int(np.prod(dims)) // 2
    L = 3 * vh
    units = np.eye(L, dtype=np.complex128).reshape(L, vh, 3)
    cols = hisq.dslash(dims, fat, lng, units, out_parity, antiperiodic_t)
    return np.ascontiguousarray(cols.reshape(L, L).T)
