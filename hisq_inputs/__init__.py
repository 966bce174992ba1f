"""Seeded synthetic inputs for the improved-staggered normal-operator solver.

This module only draws random numbers and builds input arrays (gauge links,
sources, random SU(3) matrices).  It holds none of the solver's arithmetic:
no staggered phases, no stencil, no Krylov algebra.  Both the CUDA path's tests
and the CPU oracle's tests take their inputs from here, so the two sides see
byte-identical arrays.

Recipe (stand-in for the paper's HISQ g-2 ensembles of Table 1, which are not
available): every fat link is F = exp(i*eps*H) with H = sum_a w_a lambda_a / 2,
w_a ~ N(0,1) and lambda_a the eight Gell-Mann matrices (so H is Gaussian,
traceless and Hermitian and F is in SU(3)); every long link is
G = c * exp(i*eps*H') with an independent H' and c = -1/24 (the Naik
coefficient is carried by the link data).  Sources are complex Gaussian,
Re and Im ~ N(0,1), on even sites.

Array conventions: links complex [4][V][3][3] (direction x,y,z,t, then the
lexicographic site index x + Lx*(y + Ly*(z + Lz*t)), then a 3x3 matrix with
row = colour of the result); spinor blocks complex [N][V/2][3] on one parity,
indexed by checkerboard index (lexicographic index >> 1).
"""
from __future__ import annotations

import numpy as np

LONG_COEFF = -1.0 / 24.0
EPS = 0.3


def volume(dims) -> int:
    v = 1
    for d in dims:
        v *= int(d)
    return v


def gell_mann() -> np.ndarray:
    """The eight Gell-Mann matrices, shape (8, 3, 3) complex128."""
    lam = np.zeros((8, 3, 3), dtype=np.complex128)
    lam[0][0, 1] = lam[0][1, 0] = 1
    lam[1][0, 1] = -1j
    lam[1][1, 0] = 1j
    lam[2][0, 0] = 1
    lam[2][1, 1] = -1
    lam[3][0, 2] = lam[3][2, 0] = 1
    lam[4][0, 2] = -1j
    lam[4][2, 0] = 1j
    lam[5][1, 2] = lam[5][2, 1] = 1
    lam[6][1, 2] = -1j
    lam[6][2, 1] = 1j
    lam[7][0, 0] = lam[7][1, 1] = 1 / np.sqrt(3)
    lam[7][2, 2] = -2 / np.sqrt(3)
    return lam


def _exp_i_hermitian(h: np.ndarray, eps: float) -> np.ndarray:
    """exp(i*eps*h) for a stack of Hermitian 3x3 matrices (eigendecomposition)."""
    w, q = np.linalg.eigh(h)
    ph = np.exp(1j * eps * w)
    return np.einsum("...ij,...j,...kj->...ik", q, ph, q.conj())


def random_su3(count: int, seed: int, eps: float = 1.0) -> np.ndarray:
    """count random SU(3) matrices exp(i*eps*H), H Gaussian traceless Hermitian."""
    rng = np.random.default_rng(seed)
    w = rng.standard_normal((count, 8))
    h = np.einsum("na,aij->nij", w, gell_mann() / 2)
    return _exp_i_hermitian(h, eps)


def random_links(dims, seed: int, eps: float = EPS, long_coeff: float = LONG_COEFF):
    """Fat and long links (each complex128 [4][V][3][3]) for a lattice."""
    V = volume(dims)
    rng = np.random.default_rng(seed)
    lam = gell_mann() / 2
    out = []
    for _ in range(2):
        w = rng.standard_normal((4 * V, 8))
        h = np.einsum("na,aij->nij", w, lam)
        out.append(_exp_i_hermitian(h, eps).reshape(4, V, 3, 3))
    fat, lng = out
    return np.ascontiguousarray(fat), np.ascontiguousarray(long_coeff * lng)


def gaussian_sources(dims, n_rhs: int, seed: int) -> np.ndarray:
    """n_rhs complex Gaussian even-site colour fields, complex128 [n_rhs][V/2][3]."""
    Vh = volume(dims) // 2
    rng = np.random.default_rng(seed)
    re = rng.standard_normal((n_rhs, Vh, 3))
    im = rng.standard_normal((n_rhs, Vh, 3))
    return np.ascontiguousarray(re + 1j * im)


def unit_links(dims, long_coeff: float = LONG_COEFF):
    """Free field: F = identity, G = long_coeff * identity."""
    V = volume(dims)
    eye = np.broadcast_to(np.eye(3, dtype=np.complex128), (4, V, 3, 3))
    return np.ascontiguousarray(eye), np.ascontiguousarray(long_coeff * eye)


def random_links_torch(dims, seed: int, device, eps: float = EPS, long_coeff: float = LONG_COEFF,
                       chunk: int | None = None):
    """Same recipe as random_links, drawn with torch on `device` for lattices too
    large for NumPy set-up (different random stream than random_links)."""
    import torch

    V = volume(dims)
    if chunk is None:
        chunk = (1 << 21) if torch.device(device).type == "cuda" else (1 << 22)
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    lam = torch.as_tensor(gell_mann() / 2, device=device)
    fields = []
    for _ in range(2):
        u = torch.empty((4 * V, 3, 3), dtype=torch.complex128, device=device)
        for s in range(0, 4 * V, chunk):
            e = min(4 * V, s + chunk)
            w = torch.randn((e - s, 8), generator=gen, dtype=torch.float64, device=device)
            h = torch.einsum("na,aij->nij", w.to(torch.complex128), lam)
            if torch.device(device).type == "cuda":
                # batched eigh on CUDA needs a huge workspace; the batched
                # matrix exponential of i*eps*H gives the same SU(3) matrix
                u[s:e] = torch.linalg.matrix_exp(1j * eps * h)
            else:
                ev, q = torch.linalg.eigh(h)
                ph = torch.exp(1j * eps * ev.to(torch.complex128))
                u[s:e] = torch.einsum("nij,nj,nkj->nik", q, ph, q.conj())
        fields.append(u.view(4, V, 3, 3))
    fat, lng = fields
    return fat, lng * long_coeff


def gaussian_sources_torch(dims, n_rhs: int, seed: int, device):
    import torch

    Vh = volume(dims) // 2
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    re = torch.randn((n_rhs, Vh, 3), generator=gen, dtype=torch.float64, device=device)
    im = torch.randn((n_rhs, Vh, 3), generator=gen, dtype=torch.float64, device=device)
    return torch.complex(re, im)


def batch_problems(count: int = 64, seed: int = 4000, extents=(8, 12, 16),
                   mass_range=(0.01, 0.2), n_range=(2, 16)):
    """A seeded set of independent problems for the batched solver: for each,
    a hypercubic lattice L^4 with L drawn from `extents`, a mass uniform in
    `mass_range`, a block width uniform in `n_range` (inclusive), and the seeds
    of its links and sources.  Returns a list of dicts with keys dims, mass,
    n_rhs, link_seed, source_seed."""
    rng = np.random.default_rng(seed)
    out = []
    for p in range(count):
        L = int(rng.choice(extents))
        out.append({
            "dims": (L, L, L, L),
            "mass": float(rng.uniform(*mass_range)),
            "n_rhs": int(rng.integers(n_range[0], n_range[1] + 1)),
            "link_seed": seed + 10 * p + 1,
            "source_seed": seed + 10 * p + 2,
        })
    return out
