"""GPU parity at full size: the benchmark workload (32^4, m = 0.01, N = 16)
and the large mixed-precision workload (48^3 x 96, m = 0.01, N = 32, FP16
sloppy, reliable update every 10 iterations).  The oracle cannot apply A to
whole blocks of this size quickly, so it computes sampled output sites one by
one; one column of the 32^4 solve is also solved completely by the oracle's
textbook CG and compared."""
import os

import numpy as np
import pytest

import hisq_inputs as hi
from oracle import hisq
from tests import gpu_helpers as gh
from tests import lattice_helpers as lh

pytestmark = pytest.mark.gpu

DIMS = (32, 32, 32, 32)
MASS = 0.01
N = 16


@pytest.fixture(scope="module")
def workload():
    torch = gh.torch_mod()
    fat, lng = hi.random_links_torch(DIMS, 1001, "cpu")
    b = hi.gaussian_sources(DIMS, N, 2100)
    return fat.numpy(), lng.numpy(), b


def _sample_sites(dims, count, seed):
    ev = lh.even_sites(dims) if np.prod(dims) <= 2 ** 22 else None
    rng = np.random.default_rng(seed)
    if ev is not None:
        return np.sort(rng.choice(ev, size=count, replace=False))
    # large lattice: draw coordinates and make them even
    lx, ly, lz, lt = dims
    x = rng.integers(0, lx, count)
    y = rng.integers(0, ly, count)
    z = rng.integers(0, lz, count)
    t = rng.integers(0, lt, count)
    x = x - ((x + y + z + t) & 1)
    x = np.where(x < 0, x + 2, x)
    return np.unique(x + lx * (y + ly * (z + lz * t)))


@pytest.mark.parametrize("prec", ["f64", "mixed_f32", "mixed_f16"])
def test_apply_full_size_sampled(workload, prec):
    fat, lng, b = workload
    s, _, _ = gh.make_solver(DIMS, MASS, prec=prec, links=(fat, lng), max_rhs=N)
    v = b / np.sqrt(3 * (np.prod(DIMS) // 2)) if prec == "mixed_f16" else b
    out = gh.to_np(s.apply_MdagM(v))
    sites = _sample_sites(DIMS, 48, seed=7)
    tol = gh.TOL[prec]
    for j in (0, 7, 15):
        ref = hisq.apply_A_sites(DIMS, fat, lng, MASS, v[j], sites)
        got = out[j][sites >> 1]
        assert np.abs(got - ref).max() < tol * np.abs(ref).max()


def test_solve_full_size_f64(workload):
    """The benchmark solve: true residual <= 1e-10 on sampled sites; column 0
    against the oracle's CG solution (both to 1e-12)."""
    fat, lng, b = workload
    s, _, _ = gh.make_solver(DIMS, MASS, prec="f64", links=(fat, lng), max_rhs=N)
    X, info = s.solve(b, tol=1e-10)
    assert info["status"] == 0 and info["true_rel_res_max"] <= 1e-10
    X = gh.to_np(X)
    sites = _sample_sites(DIMS, 64, seed=8)
    for j in (0, 9):
        r = b[j][sites >> 1] - hisq.apply_A_sites(DIMS, fat, lng, MASS, X[j], sites)
        rms_r = np.sqrt(np.mean(np.abs(r) ** 2))
        rms_b = np.sqrt(np.mean(np.abs(b[j][sites >> 1]) ** 2))
        assert rms_r / rms_b < 3e-10
    # solution error against the oracle at the paper's fine tolerance
    X12, info12 = s.solve(b, tol=1e-12)
    assert info12["status"] == 0
    x0, it, res = hisq.cg(DIMS, fat, lng, MASS, b[:1], tol=1e-12, max_iter=5000)
    err = np.linalg.norm(gh.to_np(X12)[0] - x0[0]) / np.linalg.norm(x0[0])
    assert err < 1e-8, err


@pytest.mark.parametrize("prec", ["mixed_f32", "mixed_f16"])
def test_solve_full_size_mixed(workload, prec):
    """The benchmark workload in the mixed forms: the search block P grows by
    orders of magnitude on this ill-conditioned problem, which must stay
    within the 16-bit storage range."""
    fat, lng, b = workload
    s, _, _ = gh.make_solver(DIMS, MASS, prec=prec, links=(fat, lng), max_rhs=N, max_iter=3000)
    X, info = s.solve(b, tol=1e-10)
    assert info["status"] == 0, info
    assert info["true_rel_res_max"] <= 1e-10
    X = gh.to_np(X)
    sites = _sample_sites(DIMS, 32, seed=10)
    r = b[3][sites >> 1] - hisq.apply_A_sites(DIMS, fat, lng, MASS, X[3], sites)
    rms_r = np.sqrt(np.mean(np.abs(r) ** 2))
    rms_b = np.sqrt(np.mean(np.abs(b[3][sites >> 1]) ** 2))
    assert rms_r / rms_b < 3e-10


def test_config_48x96_n32_mixed_f16():
    """48^3 x 96, m = 0.01, N = 32, FP16 sloppy storage, FP32 arithmetic,
    FP64 Grams / Cholesky / reliable update every 10 iterations, to 1e-10."""
    torch = gh.torch_mod()
    dims = (48, 48, 48, 96)
    n = 32
    fat, lng = hi.random_links_torch(dims, 1003, "cuda")
    b = hi.gaussian_sources_torch(dims, n, 2300, "cuda")
    gh.ensure_built()
    from paper_1710_09745_gb300 import BlockCG
    s = BlockCG(dims, fat, lng, MASS, prec="mixed_f16", max_rhs=n, ru_every=10, max_iter=5000)
    X, info = s.solve(b, tol=1e-10)
    assert info["status"] == 0, info
    assert info["true_rel_res_max"] <= 1e-10
    fat_h, lng_h = fat.cpu().numpy(), lng.cpu().numpy()
    del fat, lng
    Xh, bh = gh.to_np(X), b.cpu().numpy()
    sites = _sample_sites(dims, 16, seed=9)
    for j in (0, 31):
        r = bh[j][sites >> 1] - hisq.apply_A_sites(dims, fat_h, lng_h, MASS, Xh[j], sites)
        rms_r = np.sqrt(np.mean(np.abs(r) ** 2))
        rms_b = np.sqrt(np.mean(np.abs(bh[j][sites >> 1]) ** 2))
        assert rms_r / rms_b < 3e-10
    # column 0 against a whole oracle solve (textbook CG in FP64 to 1e-11): the
    # true residual of the full column, and the solution error, which
    # |e|/|x| <= kappa (|r_gpu| + |r_oracle|)/|b| bounds with kappa =
    # lambda_max / m^2, about 4.4e4 here (lambda_max ~ 4.3, near the free-field
    # value 4 (1 + 1/24)^2 for these smooth links)
    r0 = bh[0] - hisq.apply_A(dims, fat_h, lng_h, MASS, Xh[0])
    assert np.linalg.norm(r0) / np.linalg.norm(bh[0]) <= 1e-10
    x0, it, res = hisq.cg(dims, fat_h, lng_h, MASS, bh[:1], tol=1e-11, max_iter=5000)
    assert res[0] <= 1e-11
    err = np.linalg.norm(Xh[0] - x0[0]) / np.linalg.norm(x0[0])
    assert err < 4.4e4 * (1e-10 + 1e-11), err
    assert err < 1e-7, err
