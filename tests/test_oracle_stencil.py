"""Pins of the CPU oracle's stencil and normal operator against the
mathematics of Sec. 3.2 / Eq. 2 (not against the oracle itself)."""
import itertools

import numpy as np
import pytest

import hisq_inputs as hi
from oracle import dense, hisq
from tests import lattice_helpers as lh

C_NAIK = -1.0 / 24.0


@pytest.mark.parametrize("c", [0.0, C_NAIK])
@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (2, 4, 6, 4)])
def test_free_field_plane_waves(dims, c):
    """Unit links: A e^{ipx} = [m^2 + sum_mu (sin p + c sin 3p)^2] e^{ipx} for every p."""
    mass = 0.1
    fat, lng = hi.unit_links(dims, long_coeff=c)
    moms = [2 * np.pi * np.arange(L) / L for L in dims]
    vs, lams = [], []
    for p in itertools.product(*moms):
        vs.append(lh.plane_wave_even(dims, p, colour=len(vs) % 3))
        lams.append(lh.free_eigenvalue(p, mass, c))
    vs = np.array(vs)
    Av = hisq.apply_A(dims, fat, lng, mass, vs)
    err = np.abs(Av - np.array(lams)[:, None, None] * vs).max()
    assert err < 1e-13, err


def test_free_field_antiperiodic_t():
    """Antiperiodic in t: the t momenta become (2k+1) pi / Lt."""
    dims = (4, 4, 4, 6)
    mass = 0.05
    fat, lng = hi.unit_links(dims)
    moms = [2 * np.pi * np.arange(L) / L for L in dims[:3]] + \
        [(2 * np.arange(dims[3]) + 1) * np.pi / dims[3]]
    rng = np.random.default_rng(0)
    for p in itertools.product(*moms):
        if rng.random() > 0.3:
            continue
        v = lh.plane_wave_even(dims, p, colour=1)
        Av = hisq.apply_A(dims, fat, lng, mass, v, antiperiodic_t=True)
        lam = lh.free_eigenvalue(p, mass, C_NAIK)
        assert np.abs(Av - lam * v).max() < 1e-13


def test_free_field_with_wrong_sign_would_fail():
    """Sanity of the pin itself: the cos-spectrum of a Hermitian hopping term
    is not what the oracle produces (guards against a flipped backward sign)."""
    dims = (4, 4, 4, 4)
    mass = 0.1
    fat, lng = hi.unit_links(dims)
    p = (2 * np.pi / 4, 0.0, 2 * np.pi * 2 / 4, 2 * np.pi * 3 / 4)
    v = lh.plane_wave_even(dims, p)
    Av = hisq.apply_A(dims, fat, lng, mass, v)
    wrong = mass ** 2 + np.sum((np.cos(np.array(p)) + C_NAIK * np.cos(3 * np.array(p))) ** 2)
    assert np.abs(Av - wrong * v).max() > 1e-3


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (2, 2, 2, 2)])
def test_pure_gauge_spectrum(dims):
    """F = g(x) g(x+mu)^dag, G = c g(x) g(x+3mu)^dag: A (g v) = lambda(p) (g v)."""
    mass = 0.2
    V = int(np.prod(dims))
    g = hi.random_su3(V, seed=11)
    fat, lng = lh.pure_gauge_links(dims, g, C_NAIK)
    ge = g[lh.even_sites(dims)]
    for k, p in enumerate([(0, 0, 0, 0), (np.pi / 2, 0, np.pi, np.pi / 2),
                           (np.pi / 2, np.pi / 2, np.pi / 2, np.pi / 2)]):
        if dims[0] == 2 and any(abs(q) % np.pi > 1e-12 for q in p):
            continue
        v = lh.plane_wave_even(dims, p, colour=k % 3)
        gv = lh.apply_site_matrices(ge, v)
        Agv = hisq.apply_A(dims, fat, lng, mass, gv)
        lam = lh.free_eigenvalue(p, mass, C_NAIK)
        assert np.abs(Agv - lam * gv).max() < 1e-13


def test_gauge_covariance_random_links():
    """A'(g psi) = g (A psi) with U' = g(x) U g(x+k mu)^dag, random links and g."""
    dims = (4, 4, 4, 6)
    mass = 0.1
    V = int(np.prod(dims))
    fat, lng = hi.random_links(dims, seed=5)
    g = hi.random_su3(V, seed=6)
    fat2, lng2 = lh.gauge_transform(dims, fat, lng, g)
    psi = hi.gaussian_sources(dims, 2, seed=7)
    ge = g[lh.even_sites(dims)]
    lhs = hisq.apply_A(dims, fat2, lng2, mass, lh.apply_site_matrices(ge, psi))
    rhs = lh.apply_site_matrices(ge, hisq.apply_A(dims, fat, lng, mass, psi))
    assert np.abs(lhs - rhs).max() < 1e-12 * np.abs(rhs).max()


def test_gauge_covariance_dslash_both_parities():
    dims = (4, 4, 4, 4)
    V = int(np.prod(dims))
    fat, lng = hi.random_links(dims, seed=8)
    g = hi.random_su3(V, seed=9)
    fat2, lng2 = lh.gauge_transform(dims, fat, lng, g)
    x, y, z, t = lh.coords(dims)
    par = (x + y + z + t) & 1
    for out_p in (0, 1):
        in_sites = np.nonzero(par == 1 - out_p)[0]
        out_sites = np.nonzero(par == out_p)[0]
        psi = hi.gaussian_sources(dims, 1, seed=10 + out_p)[0]
        lhs = hisq.dslash(dims, fat2, lng2, lh.apply_site_matrices(g[in_sites], psi), out_p)
        rhs = lh.apply_site_matrices(g[out_sites], hisq.dslash(dims, fat, lng, psi, out_p))
        assert np.abs(lhs - rhs).max() < 1e-12


@pytest.mark.parametrize("antiperiodic", [False, True])
def test_hermiticity_positivity_adjointness(antiperiodic):
    dims = (4, 4, 6, 4)
    mass = 0.07
    fat, lng = hi.random_links(dims, seed=21)
    X = hi.gaussian_sources(dims, 1, seed=22)[0]
    Y = hi.gaussian_sources(dims, 1, seed=23)[0]
    AX = hisq.apply_A(dims, fat, lng, mass, X, antiperiodic)
    AY = hisq.apply_A(dims, fat, lng, mass, Y, antiperiodic)
    lhs = np.vdot(X, AY)
    rhs = np.conj(np.vdot(Y, AX))
    assert abs(lhs - rhs) < 1e-13 * abs(lhs)
    q = np.vdot(X, AX)
    assert abs(q.imag) < 1e-12 * abs(q)
    assert q.real >= mass ** 2 * np.vdot(X, X).real
    # <y_o, D_oe x_e> = -conj <x_e, D_eo y_o>
    yo = hi.gaussian_sources(dims, 1, seed=24)[0]
    lhs = np.vdot(yo, hisq.dslash(dims, fat, lng, X, 1, antiperiodic))
    rhs = -np.conj(np.vdot(X, hisq.dslash(dims, fat, lng, yo, 0, antiperiodic)))
    assert abs(lhs - rhs) < 1e-13 * abs(lhs)


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 4, 4, 4)])
def test_dense_spectrum_bounded_below(dims):
    mass = 0.1
    fat, lng = hi.random_links(dims, seed=31)
    A = dense.dense_A(dims, fat, lng, mass)
    assert np.abs(A - A.conj().T).max() < 1e-13
    w = np.linalg.eigvalsh(A)
    assert w.min() >= mass ** 2 * (1 - 1e-10)
    # D_oe = -D_eo^dag and A = m^2 - D_eo D_oe as dense matrices
    Doe = dense.dense_D(dims, fat, lng, 1)
    Deo = dense.dense_D(dims, fat, lng, 0)
    assert np.abs(Doe + Deo.conj().T).max() < 1e-13
    assert np.abs(A - (mass ** 2 * np.eye(A.shape[0]) - Deo @ Doe)).max() < 1e-12


def test_tiny_lattice_sums_coincident_hops():
    """On 2^4 every hop in direction mu reaches the same neighbour; all sixteen
    terms must still be summed.  With F = I, G = c I the forward and backward
    terms cancel pairwise, so D = 0 exactly; with F = a I (a real) they cancel
    too, but with complex scalar links F = e^{i theta} I they do not:
    D_mu = 1/2 eta (e^{i theta} - e^{-i theta}) (1 + c') per direction."""
    dims = (2, 2, 2, 2)
    V = 16
    th = 0.3
    fat = np.broadcast_to(np.exp(1j * th) * np.eye(3), (4, V, 3, 3)).copy()
    lng = np.broadcast_to(C_NAIK * np.exp(1j * th) * np.eye(3), (4, V, 3, 3)).copy()
    mass = 0.1
    # D_oe = i sin(theta) (1 + c) sum_mu eta_mu(x) (shift to the single neighbour);
    # on 2^4 D^2 restricted to even sites is -(sin th (1+c))^2 * 4 (cross terms cancel)
    v = hi.gaussian_sources(dims, 1, seed=3)[0]
    Av = hisq.apply_A(dims, fat, lng, mass, v)
    lam = mass ** 2 + 4 * (np.sin(th) * (1 + C_NAIK)) ** 2
    assert np.abs(Av - lam * v).max() < 1e-13


def test_sampled_sites_match_full_application():
    dims = (4, 4, 4, 6)
    mass = 0.03
    fat, lng = hi.random_links(dims, seed=41)
    v = hi.gaussian_sources(dims, 1, seed=42)[0]
    full = hisq.apply_A(dims, fat, lng, mass, v)
    ev = lh.even_sites(dims)
    pick = ev[[0, 5, 17, len(ev) - 1]]
    part = hisq.apply_A_sites(dims, fat, lng, mass, v, pick)
    assert np.abs(part - full[pick >> 1]).max() < 1e-14


def test_batch_problem_set_is_seeded_and_in_range():
    """The batched workload: 64 problems with L in {8, 12, 16}, m in
    [0.01, 0.2], N in 2..16, reproducible from its seed, every problem with
    its own link and source seeds."""
    import hisq_inputs as hi
    a = hi.batch_problems(64, seed=4000)
    b = hi.batch_problems(64, seed=4000)
    assert a == b
    assert len(a) == 64
    assert {p["dims"][0] for p in a} == {8, 12, 16}
    assert all(p["dims"] == (p["dims"][0],) * 4 for p in a)
    assert all(0.01 <= p["mass"] <= 0.2 for p in a)
    assert all(2 <= p["n_rhs"] <= 16 for p in a)
    seeds = [p["link_seed"] for p in a] + [p["source_seed"] for p in a]
    assert len(set(seeds)) == len(seeds)
    assert hi.batch_problems(64, seed=4001) != a
