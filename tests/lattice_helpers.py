"""Test-side lattice helpers built with NumPy index arithmetic (np.roll on a
(t, z, y, x) grid), independent of the oracle's and the kernels' own index code."""
from __future__ import annotations

import numpy as np


def grid_shape(dims):
    lx, ly, lz, lt = dims
    return (lt, lz, ly, lx)


def coords(dims):
    """Arrays x, y, z, t of shape (V,) in lexicographic order."""
    lx, ly, lz, lt = dims
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx),
                             indexing="ij")
    return x.ravel(), y.ravel(), z.ravel(), t.ravel()


def even_sites(dims):
    x, y, z, t = coords(dims)
    return np.nonzero(((x + y + z + t) & 1) == 0)[0]


def shift_index(dims, mu, k):
    """Index map i -> lexicographic index of site(i) + k*mu (periodic)."""
    V = int(np.prod(dims))
    idx = np.arange(V).reshape(grid_shape(dims))
    axis = 3 - mu
    return np.roll(idx, -k, axis=axis).ravel()


def gauge_transform(dims, fat, lng, g):
    """U'_mu(x) = g(x) U_mu(x) g(x+k mu)^dag for k=1 (fat) and k=3 (long)."""
    fat2 = np.empty_like(fat)
    lng2 = np.empty_like(lng)
    gd = g.conj().transpose(0, 2, 1)
    for mu in range(4):
        s1 = shift_index(dims, mu, 1)
        s3 = shift_index(dims, mu, 3)
        fat2[mu] = g @ fat[mu] @ gd[s1]
        lng2[mu] = g @ lng[mu] @ gd[s3]
    return fat2, lng2


def pure_gauge_links(dims, g, c):
    """F_mu(x) = g(x) g(x+mu)^dag, G_mu(x) = c g(x) g(x+3mu)^dag."""
    V = int(np.prod(dims))
    fat = np.empty((4, V, 3, 3), dtype=np.complex128)
    lng = np.empty((4, V, 3, 3), dtype=np.complex128)
    gd = g.conj().transpose(0, 2, 1)
    for mu in range(4):
        fat[mu] = g @ gd[shift_index(dims, mu, 1)]
        lng[mu] = c * (g @ gd[shift_index(dims, mu, 3)])
    return fat, lng


def plane_wave_even(dims, p, colour=0):
    """v(x) = exp(i p.x) e_colour on even sites, as a [V/2][3] block."""
    x, y, z, t = coords(dims)
    ev = even_sites(dims)
    phase = np.exp(1j * (p[0] * x + p[1] * y + p[2] * z + p[3] * t))[ev]
    v = np.zeros((len(ev), 3), dtype=np.complex128)
    v[:, colour] = phase
    return v


def free_eigenvalue(p, mass, c):
    """m^2 + sum_mu (sin p_mu + c sin 3 p_mu)^2."""
    p = np.asarray(p, dtype=np.float64)
    return mass * mass + np.sum((np.sin(p) + c * np.sin(3 * p)) ** 2)


def apply_site_matrices(g_even, v):
    """(g v)(x) for x even: g_even [V/2][3][3], v [..., V/2, 3]."""
    return np.einsum("sab,...sb->...sa", g_even, v)
