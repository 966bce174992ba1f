"""Pins of the oracle's link gradient (oracle_link_grad) against central
finite differences of the loss, computed with dense solves on 4^4.

The loss L(U) = Re sum_i c_i^dag A(U)^-1 phi_i covers both the self-adjoint
case (c = phi: L = sum_i phi_i^dag A^-1 phi_i, the adjoint block equals the
solution) and a general one (c independent: the adjoint block A^-1 c differs).
The gradient convention is G = dL/dRe(u) + i dL/dIm(u) per link entry u, so a
perturbation u -> u + h gives dL/dh = Re G and u -> u + i h gives Im G; along
a direction dU over all links, dL/dh = Re sum conj(G) dU."""
import numpy as np
import pytest

import hisq_inputs as hi
from oracle import hisq
from oracle.dense import dense_A

DIMS = (4, 4, 4, 4)
MASS = 0.1
H = 1e-6


def _loss(fat, lng, phi, c, antiperiodic):
    A = dense_A(DIMS, fat, lng, MASS, antiperiodic)
    n = phi.shape[0]
    X = np.linalg.solve(A, phi.reshape(n, -1).T).T
    return float(np.real(np.sum(np.conj(c.reshape(n, -1)) * X)))


def _setup(self_adjoint, antiperiodic, seed=11):
    fat, lng = hi.random_links(DIMS, seed)
    phi = hi.gaussian_sources(DIMS, 2, seed + 1)
    c = phi if self_adjoint else hi.gaussian_sources(DIMS, 2, seed + 2)
    A = dense_A(DIMS, fat, lng, MASS, antiperiodic)
    n = phi.shape[0]
    x = np.linalg.solve(A, phi.reshape(n, -1).T).T.reshape(phi.shape)
    lam = np.linalg.solve(A.conj().T, c.reshape(n, -1).T).T.reshape(phi.shape)
    gf, gl = hisq.link_grad(DIMS, fat, lng, x, lam, antiperiodic)
    return fat, lng, phi, c, gf, gl


def _sample_entries(rng, count):
    """Link entries (which, mu, site, a, b): both parities, every direction,
    and sites on the t boundary (whose hops cross it)."""
    V = int(np.prod(DIMS))
    out = []
    for k in range(count):
        which = k % 2
        mu = (k // 2) % 4
        if k % 3 == 0:  # t = Lt - 1 (and Lt - 3 for the long hop): boundary-crossing hops
            t = DIMS[3] - 1 - (2 * which if k % 2 else 0)
            xs = rng.integers(0, DIMS[0], 3)
            site = int(xs[0] + DIMS[0] * (xs[1] + DIMS[1] * (xs[2] + DIMS[2] * t)))
        else:
            site = int(rng.integers(0, V))
        out.append((which, mu, site, int(rng.integers(0, 3)), int(rng.integers(0, 3))))
    return out


@pytest.mark.parametrize("self_adjoint", [True, False])
@pytest.mark.parametrize("antiperiodic", [False, True])
def test_link_grad_entries_match_central_differences(self_adjoint, antiperiodic):
    fat, lng, phi, c, gf, gl = _setup(self_adjoint, antiperiodic)
    scale = max(np.abs(gf).max(), np.abs(gl).max())
    rng = np.random.default_rng(5)
    parities = set()
    for which, mu, site, a, b in _sample_entries(rng, 16):
        G = (gl if which else gf)[mu, site, a, b]
        for part, step in ((0, H), (1, 1j * H)):
            Up = [fat.copy(), lng.copy()]
            Um = [fat.copy(), lng.copy()]
            Up[which][mu, site, a, b] += step
            Um[which][mu, site, a, b] -= step
            fd = (_loss(Up[0], Up[1], phi, c, antiperiodic) -
                  _loss(Um[0], Um[1], phi, c, antiperiodic)) / (2 * H)
            ref = G.real if part == 0 else G.imag
            # rounding of the FD quotient ~ 1e-16 |L| / h; |L| <~ 1e4 here
            assert abs(fd - ref) <= 2e-6 * scale, (which, mu, site, a, b, part, fd, ref)
        x = np.unravel_index(site, DIMS[::-1])
        parities.add(sum(x) & 1)
    assert parities == {0, 1}


@pytest.mark.parametrize("self_adjoint", [True, False])
def test_link_grad_directional_derivative(self_adjoint):
    """A random direction through all links at once: a dropped term, wrong
    sign or transposed factor anywhere in the gradient changes the result."""
    fat, lng, phi, c, gf, gl = _setup(self_adjoint, False, seed=21)
    rng = np.random.default_rng(9)
    dF = rng.standard_normal(fat.shape) + 1j * rng.standard_normal(fat.shape)
    dL = rng.standard_normal(lng.shape) + 1j * rng.standard_normal(lng.shape)
    fd = (_loss(fat + H * dF, lng + H * dL, phi, c, False) -
          _loss(fat - H * dF, lng - H * dL, phi, c, False)) / (2 * H)
    pred = float(np.real(np.sum(np.conj(gf) * dF) + np.sum(np.conj(gl) * dL)))
    assert abs(fd - pred) <= 1e-6 * abs(pred), (fd, pred)
    # and the fat and long parts separately
    fd_f = (_loss(fat + H * dF, lng, phi, c, False) - _loss(fat - H * dF, lng, phi, c, False)) / (2 * H)
    pred_f = float(np.real(np.sum(np.conj(gf) * dF)))
    assert abs(fd_f - pred_f) <= 1e-6 * abs(pred_f), (fd_f, pred_f)


def test_link_grad_tiny_lattice_coincident_hops():
    """2^4: the +-1 and +-3 hops reach the same neighbours; every link term
    still counts once.  Checked along a random direction."""
    dims = (2, 2, 2, 2)
    fat, lng = hi.random_links(dims, 31)
    phi = hi.gaussian_sources(dims, 1, 32)
    A = dense_A(dims, fat, lng, MASS)
    x = np.linalg.solve(A, phi.reshape(1, -1).T).T.reshape(phi.shape)
    gf, gl = hisq.link_grad(dims, fat, lng, x, x)
    rng = np.random.default_rng(3)
    dF = rng.standard_normal(fat.shape) + 1j * rng.standard_normal(fat.shape)

    def loss(f):
        Ad = dense_A(dims, f, lng, MASS)
        return float(np.real(np.vdot(phi.reshape(-1), np.linalg.solve(Ad, phi.reshape(-1)))))

    fd = (loss(fat + H * dF) - loss(fat - H * dF)) / (2 * H)
    pred = float(np.real(np.sum(np.conj(gf) * dF)))
    assert abs(fd - pred) <= 1e-6 * abs(pred)
