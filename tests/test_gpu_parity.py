"""GPU parity: the CUDA path through the C ABI against the CPU oracle,
element by element, on seeded inputs that span several CTAs and a ragged
tail; edge cases of the method; full-size sampled checks."""
import numpy as np
import pytest

import hisq_inputs as hi
from oracle import block as oblock
from oracle import hisq
from tests import gpu_helpers as gh
from tests import lattice_helpers as lh

pytestmark = pytest.mark.gpu

DIMS = (6, 8, 10, 12)   # Vh = 2880: several CTAs and a ragged last one
PRECS = ["f64", "f64_native", "mixed_f32"]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("N", [1, 3, 4, 16])
@pytest.mark.parametrize("parity", [0, 1])
def test_dslash_parity(prec, N, parity):
    s, fat, lng = gh.make_solver(DIMS, 0.1, prec=prec, seed=1001)
    psi = hi.gaussian_sources(DIMS, N, seed=77 + N)
    out = gh.to_np(s.dslash(psi, parity))
    ref = hisq.dslash(DIMS, fat, lng, psi, parity)
    assert gh.rel_err(out, ref) < gh.TOL[prec]


TMA = 256
ASYNC = 512
BLOCKED = 4096  # plain kernel, persistent grid of contiguous site ranges


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("variant", [1, 2, 4, 8, TMA + 1, TMA + 2, TMA + 4, TMA + 8,
                                     ASYNC + 1, ASYNC + 2, ASYNC + 4, ASYNC + 8,
                                     BLOCKED + 1, BLOCKED + 4, BLOCKED + 8])
@pytest.mark.parametrize("N,parity", [(2, 0), (5, 1), (16, 0), (16, 1), (33, 1)])
def test_dslash_every_kernel_variant(prec, variant, N, parity):
    """Each stencil kernel (register tile R; plain, bulk-copy pipelined or
    cp.async prefetching) against the oracle; unsupported pipelined cases
    fall back to the plain kernel."""
    s, fat, lng = gh.make_solver(DIMS, 0.1, prec=prec, seed=1011, max_rhs=max(N, 16),
                                 dslash_variant=variant)
    psi = hi.gaussian_sources(DIMS, N, seed=99 + N)
    out = gh.to_np(s.dslash(psi, parity))
    ref = hisq.dslash(DIMS, fat, lng, psi, parity)
    assert gh.rel_err(out, ref) < gh.TOL[prec]


@pytest.mark.parametrize("variant", [TMA + 2, TMA + 4, ASYNC + 2, ASYNC + 4])
def test_solve_with_pipelined_stencil(variant):
    dims = (8, 8, 8, 8)
    s, fat, lng = gh.make_solver(dims, 0.05, seed=1012, max_rhs=8, dslash_variant=variant)
    b = hi.gaussian_sources(dims, 8, seed=2012)
    X, info = s.solve(b, tol=1e-10)
    assert info["status"] == 0
    r = b - hisq.apply_A(dims, fat, lng, 0.05, gh.to_np(X))
    rel = np.linalg.norm(r.reshape(8, -1), axis=1) / np.linalg.norm(b.reshape(8, -1), axis=1)
    assert rel.max() <= 1e-10


PRECS16 = ["mixed_f16", "mixed_bf16"]


@pytest.mark.parametrize("prec", PRECS16)
@pytest.mark.parametrize("variant", [0, 1, 2, 4, 8, TMA + 4, ASYNC + 4,
                                     BLOCKED + 4])
@pytest.mark.parametrize("N,parity", [(1, 0), (3, 1), (8, 0), (16, 1)])
def test_dslash_16bit(prec, variant, N, parity):
    """16-bit storage with FP32 arithmetic; inputs at the magnitude of the
    solver's normalised block vectors."""
    s, fat, lng = gh.make_solver(DIMS, 0.1, prec=prec, seed=1013, max_rhs=16,
                                 dslash_variant=variant)
    psi = hi.gaussian_sources(DIMS, N, seed=120 + N) / np.sqrt(3 * psi_sites(DIMS))
    out = gh.to_np(s.dslash(psi, parity))
    ref = hisq.dslash(DIMS, fat, lng, psi, parity)
    assert gh.rel_err(out, ref) < gh.TOL[prec]


def psi_sites(dims):
    return int(np.prod(dims)) // 2


@pytest.mark.parametrize("prec", PRECS16)
def test_apply_and_blas_16bit(prec):
    N = 8
    s, fat, lng = gh.make_solver(DIMS, 0.05, prec=prec, seed=1014, max_rhs=N)
    sc = 1.0 / np.sqrt(3 * psi_sites(DIMS))
    v = hi.gaussian_sources(DIMS, N, seed=130) * sc
    w = hi.gaussian_sources(DIMS, N, seed=131) * sc
    assert gh.rel_err(gh.to_np(s.apply_MdagM(v)), hisq.apply_A(DIMS, fat, lng, 0.05, v)) < gh.TOL[prec]
    K = gh.to_np(s.block_cdot(v, w))
    Kref = oblock.block_cdot(oblock.as_columns(v), oblock.as_columns(w))
    assert np.abs(K - Kref).max() < gh.TOL[prec] * 0.1
    Q, R = s.thin_qr(v)
    Qr, Rr = oblock.thin_qr(oblock.as_columns(v))
    assert gh.rel_err(gh.to_np(R), Rr) < gh.TOL[prec]


@pytest.mark.parametrize("prec", PRECS16)
def test_solve_16bit_reliable_updates(prec):
    """Sloppy 16-bit iterations, FP64 reliable updates: the true residual still
    reaches 1e-10 (Algorithm 3)."""
    dims = (8, 8, 8, 8)
    mass = 0.05
    s, fat, lng = gh.make_solver(dims, mass, prec=prec, seed=1015, max_rhs=8)
    b = hi.gaussian_sources(dims, 8, seed=2015)
    X, info = s.solve(b, tol=1e-10)
    assert info["status"] == 0, info
    r = b - hisq.apply_A(dims, fat, lng, mass, gh.to_np(X))
    rel = np.linalg.norm(r.reshape(8, -1), axis=1) / np.linalg.norm(b.reshape(8, -1), axis=1)
    assert rel.max() <= 1e-10
    Xc, ic = s.solve_cg(b[:2], tol=1e-10)
    assert ic["status"] == 0, ic
    rc = b[:2] - hisq.apply_A(dims, fat, lng, mass, gh.to_np(Xc))
    relc = np.linalg.norm(rc.reshape(2, -1), axis=1) / np.linalg.norm(b[:2].reshape(2, -1), axis=1)
    assert relc.max() <= 1e-10


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("N", [1, 5, 8])
@pytest.mark.parametrize("antiperiodic", [False, True])
def test_apply_MdagM_parity(prec, N, antiperiodic):
    s, fat, lng = gh.make_solver(DIMS, 0.05, prec=prec, seed=1002, antiperiodic_t=antiperiodic)
    v = hi.gaussian_sources(DIMS, N, seed=88)
    out = gh.to_np(s.apply_MdagM(v))
    ref = hisq.apply_A(DIMS, fat, lng, 0.05, v, antiperiodic)
    assert gh.rel_err(out, ref) < gh.TOL[prec]


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (2, 4, 2, 6), (4, 4, 4, 4)])
def test_apply_tiny_lattices_wraparound(dims):
    """On 2^4 and 4^4 forward/backward and 1/3-hop neighbours coincide; every
    term must still be summed."""
    s, fat, lng = gh.make_solver(dims, 0.1, prec="f64", seed=1003, max_rhs=4)
    v = hi.gaussian_sources(dims, 4, seed=5)
    assert gh.rel_err(gh.to_np(s.apply_MdagM(v)), hisq.apply_A(dims, fat, lng, 0.1, v)) < 1e-12


def test_free_field_plane_wave_on_gpu():
    dims = (8, 8, 8, 8)
    fat, lng = hi.unit_links(dims)
    s, _, _ = gh.make_solver(dims, 0.2, links=(fat, lng), max_rhs=2)
    p = (2 * np.pi / 8, 3 * 2 * np.pi / 8, 0.0, 5 * 2 * np.pi / 8)
    v = lh.plane_wave_even(dims, p, colour=2)
    out = gh.to_np(s.apply_MdagM(v))[0]
    lam = lh.free_eigenvalue(p, 0.2, hi.LONG_COEFF)
    assert np.abs(out - lam * v).max() < 1e-12


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("N", [1, 4, 16, 33])
def test_block_cdot_parity(prec, N):
    s, _, _ = gh.make_solver(DIMS, 0.1, prec=prec, max_rhs=max(N, 16))
    X = hi.gaussian_sources(DIMS, N, seed=9)
    Y = hi.gaussian_sources(DIMS, N, seed=10)
    K = gh.to_np(s.block_cdot(X, Y))
    Kref = oblock.block_cdot(oblock.as_columns(X), oblock.as_columns(Y))
    scale = np.linalg.norm(oblock.as_columns(X), axis=0).max() * np.linalg.norm(oblock.as_columns(Y), axis=0).max()
    tol = {"f64": 1e-13, "f64_native": 1e-14, "mixed_f32": 1e-5}[prec]
    assert np.abs(K - Kref).max() < tol * scale


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("N", [1, 6, 16, 64])
def test_block_caxpy_parity(prec, N):
    s, _, _ = gh.make_solver((4, 4, 4, 6), 0.1, prec=prec, max_rhs=max(N, 16))
    X = hi.gaussian_sources((4, 4, 4, 6), N, seed=11)
    Y = hi.gaussian_sources((4, 4, 4, 6), N, seed=12)
    rng = np.random.default_rng(13)
    a = rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))
    out = gh.to_np(s.block_caxpy(X, a, Y))
    ref = oblock.from_columns(oblock.block_caxpy(oblock.as_columns(Y), oblock.as_columns(X), a), X.shape[1])
    tol = {"f64": 1e-13, "f64_native": 1e-14, "mixed_f32": 1e-5}[prec]
    assert gh.rel_err(out, ref) < tol * np.sqrt(N)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("N", [1, 7, 16, 64])
def test_thin_qr_parity(prec, N):
    dims = (4, 4, 6, 8)
    s, _, _ = gh.make_solver(dims, 0.1, prec=prec, max_rhs=max(N, 16))
    M = hi.gaussian_sources(dims, N, seed=14)
    Q, R = s.thin_qr(M)
    Q, R = gh.to_np(Q), gh.to_np(R)
    Qr, Rr = oblock.thin_qr(oblock.as_columns(M))
    tol = {"f64": 1e-12, "f64_native": 1e-13, "mixed_f32": 1e-4}[prec]
    assert gh.rel_err(R, Rr) < tol
    Qc = oblock.as_columns(Q)
    assert np.abs(Qc.conj().T @ Qc - np.eye(N)).max() < 10 * tol


def test_thin_qr_breakdown_on_dependent_columns():
    from paper_1710_09745_gb300 import BlockCGError
    dims = (4, 4, 4, 4)
    s, _, _ = gh.make_solver(dims, 0.1, max_rhs=4)
    M = hi.gaussian_sources(dims, 3, seed=15)
    M[2] = M[0]
    with pytest.raises(BlockCGError) as e:
        s.thin_qr(M)
    assert e.value.status == 4


# ------------------------------------------------------------------ solvers
def _oracle_solution(dims, fat, lng, mass, b):
    x, _, res = hisq.cg(dims, fat, lng, mass, b, tol=1e-13)
    return x


def test_solve_config_4x4_n4():
    """4^4, m = 0.1, N = 4, FP64 block CG to 1e-10."""
    dims = (4, 4, 4, 4)
    s, fat, lng = gh.make_solver(dims, 0.1, seed=1001, max_rhs=4)
    b = hi.gaussian_sources(dims, 4, seed=2001)
    X, info = s.solve(b, tol=1e-10)
    X = gh.to_np(X)
    assert info["status"] == 0, info
    r = b - hisq.apply_A(dims, fat, lng, 0.1, X)
    rel = np.linalg.norm(r.reshape(4, -1), axis=1) / np.linalg.norm(b.reshape(4, -1), axis=1)
    assert rel.max() <= 1e-10, rel
    assert info["true_rel_res_max"] <= 1e-10
    xo = _oracle_solution(dims, fat, lng, 0.1, b)
    err = np.linalg.norm((X - xo).reshape(4, -1), axis=1) / np.linalg.norm(xo.reshape(4, -1), axis=1)
    assert err.max() < 1e-8, err


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("N", [1, 8])
def test_solve_against_oracle(prec, N):
    dims = (8, 8, 8, 8)
    mass = 0.05
    s, fat, lng = gh.make_solver(dims, mass, prec=prec, seed=1005, max_rhs=8)
    b = hi.gaussian_sources(dims, N, seed=2005)
    X, info = s.solve(b, tol=1e-12)
    X = gh.to_np(X)
    assert info["status"] == 0, info
    r = b - hisq.apply_A(dims, fat, lng, mass, X)
    rel = np.linalg.norm(r.reshape(N, -1), axis=1) / np.linalg.norm(b.reshape(N, -1), axis=1)
    assert rel.max() <= 1e-12 * 1.01, rel
    xo = _oracle_solution(dims, fat, lng, mass, b)
    err = np.linalg.norm((X - xo).reshape(N, -1), axis=1) / np.linalg.norm(xo.reshape(N, -1), axis=1)
    assert err.max() < 1e-8, err


@pytest.mark.parametrize("prec", ["f64", "f64_native"])
def test_solve_cg_against_oracle(prec):
    dims = (8, 8, 8, 8)
    mass = 0.05
    s, fat, lng = gh.make_solver(dims, mass, prec=prec, seed=1006, max_rhs=4)
    b = hi.gaussian_sources(dims, 3, seed=2006)
    X, info = s.solve_cg(b, tol=1e-12)
    X = gh.to_np(X)
    assert info["status"] == 0, info
    xo, iters, _ = hisq.cg(dims, fat, lng, mass, b, tol=1e-12)
    err = np.linalg.norm((X - xo).reshape(3, -1), axis=1) / np.linalg.norm(xo.reshape(3, -1), axis=1)
    assert err.max() < 1e-8
    # same algorithm (reliable updates keep the search direction), same
    # stopping rule: iteration counts agree to a few percent
    assert abs(info["iters"] - int(iters.sum())) <= 0.05 * int(iters.sum()) + 3


def test_block_fewer_iterations_than_cg():
    dims = (8, 8, 8, 8)
    s, _, _ = gh.make_solver(dims, 0.01, seed=1007, max_rhs=8)
    b = hi.gaussian_sources(dims, 8, seed=2007)
    _, ib = s.solve(b, tol=1e-10)
    _, ic = s.solve_cg(b[:2], tol=1e-10)
    assert ib["status"] == 0 and ic["status"] == 0
    assert ib["iters"] < ic["iters"] / 2


def test_solve_initial_guess_and_resume():
    """Alg. 1 starts from any X: resuming from a partial solve converges."""
    dims = (6, 6, 6, 6)
    s, fat, lng = gh.make_solver(dims, 0.1, seed=1008, max_rhs=4, max_iter=5)
    b = hi.gaussian_sources(dims, 4, seed=2008)
    X1, i1 = s.solve(b, tol=1e-10)
    assert i1["status"] == 6           # not converged after 5 iterations
    assert 1e-10 < i1["true_rel_res_max"] < 1.0
    s2, _, _ = gh.make_solver(dims, 0.1, seed=1008, max_rhs=4)
    X2, i2 = s2.solve(b, X0=X1, tol=1e-10)
    assert i2["status"] == 0
    r = b - hisq.apply_A(dims, fat, lng, 0.1, gh.to_np(X2))
    assert (np.linalg.norm(r.reshape(4, -1), axis=1) / np.linalg.norm(b.reshape(4, -1), axis=1)).max() <= 1e-10


def test_solve_dependent_rhs_breaks_down():
    from paper_1710_09745_gb300 import BlockCGError
    dims = (4, 4, 4, 4)
    s, _, _ = gh.make_solver(dims, 0.1, max_rhs=4)
    b = hi.gaussian_sources(dims, 3, seed=16)
    b[1] = 2.0 * b[0]
    with pytest.raises(BlockCGError) as e:
        s.solve(b, tol=1e-10)
    assert e.value.status == 4


def test_solve_zero_rhs_rejected():
    from paper_1710_09745_gb300 import BlockCGError
    dims = (4, 4, 4, 4)
    s, _, _ = gh.make_solver(dims, 0.1, max_rhs=4)
    b = hi.gaussian_sources(dims, 2, seed=17)
    b[1] = 0
    with pytest.raises(BlockCGError):
        s.solve(b, tol=1e-10)


def test_nonfinite_source_reported():
    from paper_1710_09745_gb300 import BlockCGError
    dims = (4, 4, 4, 4)
    s, _, _ = gh.make_solver(dims, 0.1, max_rhs=4)
    b = hi.gaussian_sources(dims, 2, seed=18)
    b[0, 3, 1] = np.nan
    with pytest.raises(BlockCGError) as e:
        s.solve(b, tol=1e-10)
    assert e.value.status == 5


def test_bad_arguments():
    from paper_1710_09745_gb300 import BlockCGError
    dims = (4, 4, 4, 4)
    s, _, _ = gh.make_solver(dims, 0.1, max_rhs=4)
    b = hi.gaussian_sources(dims, 5, seed=19)
    with pytest.raises(BlockCGError):
        s.solve(b, tol=1e-10)          # more RHS than the workspace holds
    with pytest.raises(BlockCGError):
        s.solve(b[:2], tol=0.0)


def test_mixed_precision_reliable_updates():
    dims = (8, 8, 8, 8)
    mass = 0.02
    s, fat, lng = gh.make_solver(dims, mass, prec="mixed_f32", seed=1009, max_rhs=8)
    b = hi.gaussian_sources(dims, 8, seed=2009)
    X, info = s.solve(b, tol=1e-10)
    assert info["status"] == 0
    assert info["reliable_updates"] >= 3
    r = b - hisq.apply_A(dims, fat, lng, mass, gh.to_np(X))
    rel = np.linalg.norm(r.reshape(8, -1), axis=1) / np.linalg.norm(b.reshape(8, -1), axis=1)
    assert rel.max() <= 1e-10
    s64, _, _ = gh.make_solver(dims, mass, prec="f64", seed=1009, max_rhs=8)
    _, i64 = s64.solve(b, tol=1e-10)
    assert info["iters"] <= 1.6 * i64["iters"]


def test_max_rhs_64():
    dims = (4, 4, 4, 8)
    s, fat, lng = gh.make_solver(dims, 0.2, seed=1010, max_rhs=64)
    b = hi.gaussian_sources(dims, 64, seed=2010)
    X, info = s.solve(b, tol=1e-10)
    assert info["status"] == 0
    r = b - hisq.apply_A(dims, fat, lng, 0.2, gh.to_np(X))
    rel = np.linalg.norm(r.reshape(64, -1), axis=1) / np.linalg.norm(b.reshape(64, -1), axis=1)
    assert rel.max() <= 1e-10


def test_solve_in_place_out_matches_allocating_solve():
    """solve(..., out=T) uses T as the initial guess and writes X into it: the
    result equals the allocating call bit for bit, and X0 is copied into out."""
    import torch
    s, fat, lng = gh.make_solver((4, 4, 4, 4), 0.1, prec="f64", seed=1090, max_rhs=4)
    b = torch.as_tensor(hi.gaussian_sources((4, 4, 4, 4), 3, 2090)).cuda()
    X1, i1 = s.solve(b, tol=1e-10)
    out = torch.zeros_like(b)
    X2, i2 = s.solve(b, tol=1e-10, out=out)
    assert X2.data_ptr() == out.data_ptr()
    assert torch.equal(X1, X2) and i1["iters"] == i2["iters"]
    # a converged initial guess copied in through X0: no iterations needed
    out2 = torch.empty_like(b)
    X3, i3 = s.solve(b, X0=X1, tol=1e-10, out=out2)
    assert X3.data_ptr() == out2.data_ptr() and i3["iters"] == 0
    with pytest.raises(ValueError):
        s.solve(b, out=torch.zeros((2, b.shape[1], 3), dtype=b.dtype, device=b.device))


@pytest.mark.parametrize("prec,N,dims", [("mixed_f32", 64, (4, 4, 4, 8)),
                                          ("mixed_f32", 24, (4, 4, 4, 8)),
                                          ("f64_native", 40, (8, 8, 4, 8))])
def test_solve_wide_blocks_double_buffered_update(prec, N, dims):
    """Wide blocks in the storage kinds whose fused update double-buffers its
    tiles: small tiles (4 sites at N = 64) and several coefficient chunks.
    The native-FP64 case runs on 8x8x4x8 (L = 3072 rows): on 4x4x4x8 (L = 768)
    forty columns exhaust the space after L/N ~ 19 iterations and the block
    breaks down in exact arithmetic too (the oracle's block CG reaches a
    relative Cholesky pivot of 2e-14 there), which the solver reports as
    BLOCKCG_ERR_BREAKDOWN."""
    s, fat, lng = gh.make_solver(dims, 0.2, prec=prec, seed=1011, max_rhs=N)
    b = hi.gaussian_sources(dims, N, seed=2011)
    X, info = s.solve(b, tol=1e-10)
    assert info["status"] == 0, info
    r = b - hisq.apply_A(dims, fat, lng, 0.2, gh.to_np(X))
    rel = np.linalg.norm(r.reshape(N, -1), axis=1) / np.linalg.norm(b.reshape(N, -1), axis=1)
    assert rel.max() <= 1.05e-10


def _oracle_rel_res(dims, fat, lng, mass, b, X):
    r = b - hisq.apply_A(dims, fat, lng, mass, X)
    n = b.shape[0]
    return np.linalg.norm(r.reshape(n, -1), axis=1) / np.linalg.norm(b.reshape(n, -1), axis=1)


@pytest.mark.parametrize("prec", ["f64", "mixed_f32", "mixed_f16"])
def test_per_rhs_true_residuals_match_oracle(prec):
    """blockcg_stats.true_rel_res: the library's per-column true relative
    residual |b_i - A x_i| / |b_i| at exit against the oracle's, recomputed in
    FP64 on the CPU from the returned X.  Both are FP64 computations of a
    residual ~1e-10 |b|, so they agree to ~1e-15 |b| (absolute, relative to
    |b_i|), not to a relative 1e-15."""
    dims, mass, N = (8, 8, 8, 8), 0.05, 6
    s, fat, lng = gh.make_solver(dims, mass, prec=prec, seed=1021, max_rhs=8)
    b = hi.gaussian_sources(dims, N, seed=2021)
    X, info = s.solve(b, tol=1e-10)
    assert info["status"] == 0
    ref = _oracle_rel_res(dims, fat, lng, mass, b, gh.to_np(X))
    got = np.array(info["true_rel_res"])
    assert got.shape == (N,) and np.isfinite(got).all()
    assert np.abs(got - ref).max() < 1e-13
    assert abs(got.max() - info["true_rel_res_max"]) < 1e-15
    assert got.max() <= 1e-10
    # the CG baseline fills the same array, column by column
    Xc, ic = s.solve_cg(b[:3], tol=1e-10)
    refc = _oracle_rel_res(dims, fat, lng, mass, b[:3], gh.to_np(Xc))
    assert np.abs(np.array(ic["true_rel_res"]) - refc).max() < 1e-13


def test_bulk_copy_wait_limit_reports_timeout_and_context_survives():
    """A bounded device wait that runs out: the bulk-copy stencil with a
    1 ns wait limit gives up on its first stage, waits for every copy it has
    issued, records BLOCKCG_ERR_TIMEOUT and returns; the solve reports it and
    the context stays usable (a normal solve follows)."""
    dims, mass, N = (8, 8, 8, 8), 0.05, 4
    s, fat, lng = gh.make_solver(dims, mass, seed=1022, max_rhs=4, dslash_variant=TMA + 2,
                                 wait_limit_ns=1)
    b = hi.gaussian_sources(dims, N, seed=2022)
    from paper_1710_09745_gb300 import BlockCGError
    with pytest.raises(BlockCGError) as ei:
        s.solve(b, tol=1e-10)
    assert ei.value.status == 7
    s.close()
    s2, fat, lng = gh.make_solver(dims, mass, seed=1022, max_rhs=4, dslash_variant=TMA + 2)
    X, info2 = s2.solve(b, tol=1e-10)
    assert info2["status"] == 0
    assert _oracle_rel_res(dims, fat, lng, mass, b, gh.to_np(X)).max() <= 1e-10


def test_tune_then_solve_uses_the_tuned_kernel():
    """blockcg_tune runs the autotuner ahead of the solve; the solve then
    reports the tuned kernel and converges as usual."""
    dims, mass, N = (8, 8, 8, 8), 0.05, 8
    s, fat, lng = gh.make_solver(dims, mass, seed=1023, max_rhs=8)
    s.tune(N)
    b = hi.gaussian_sources(dims, N, seed=2023)
    X, info = s.solve(b, tol=1e-10)
    assert info["status"] == 0 and info["stencil_variant"] != 0
    assert _oracle_rel_res(dims, fat, lng, mass, b, gh.to_np(X)).max() <= 1e-10


def test_solve_many_picks_width_and_persists_it(tmp_path):
    """blockcg_solve_many with width 0 on 40 right-hand sides: the first
    blocks are solved at the candidate widths 8 and 16 (32 no longer fits the
    remaining 16), the rest at the faster one; every column meets the
    tolerance on the oracle's residual; the choice is written to the cache
    file, and a second handle naming the file reuses it without exploring."""
    dims, mass, M = (8, 8, 8, 8), 0.05, 40
    cache = tmp_path / "tune.json"
    s, fat, lng = gh.make_solver(dims, mass, seed=1024, max_rhs=32)
    s.set_tune_cache(cache)
    b = hi.gaussian_sources(dims, M, seed=2024)
    X, info = s.solve_many(b, tol=1e-10)
    assert info["status"] == 0, info
    assert sorted(info["candidates"]) == [8, 16]
    assert info["width"] in (8, 16)
    assert info["blocks"] == 2 + (16 + info["width"] - 1) // info["width"]
    ref = _oracle_rel_res(dims, fat, lng, mass, b, gh.to_np(X))
    assert ref.max() <= 1e-10
    assert np.abs(np.array(info["true_rel_res"]) - ref).max() < 1e-13
    text = cache.read_text()
    assert '"width/8.8.8.8/' in text and '"stencil/8.8.8.8/' in text
    s2, _, _ = gh.make_solver(dims, mass, seed=1024, max_rhs=32)
    s2.set_tune_cache(cache)
    X2, info2 = s2.solve_many(b[:24], tol=1e-10)
    assert info2["status"] == 0 and info2["from_cache"] == 1
    assert info2["width"] == info["width"] and info2["candidates"] == {}
    assert _oracle_rel_res(dims, fat, lng, mass, b[:24], gh.to_np(X2)).max() <= 1e-10
    # a fixed width needs no cache
    X3, info3 = s.solve_many(b[:10], tol=1e-10, width=4)
    assert info3["blocks"] == 3 and info3["width"] == 4
    assert _oracle_rel_res(dims, fat, lng, mass, b[:10], gh.to_np(X3)).max() <= 1e-10


@pytest.mark.parametrize("prec,kind", [("mixed_f32", 1), ("mixed_f16", 3)])
@pytest.mark.parametrize("upd", [4, 8 | 64, 8 | 128, 16 | 64 | 128, 32])
def test_forced_blas_tiles_converge(tmp_path, prec, kind, upd):
    """Every shape the block-BLAS tile tuner can choose, forced through the
    tuning cache (sites per tile of the fused update, one or two rows per
    thread (64), X staged or read from global memory (128); Gram tiles of 16
    and 32 sites): each solve meets tol on the oracle's residual."""
    import json
    torch = gh.torch_mod()
    dims, mass, N = (8, 8, 8, 8), 0.05, 8
    dev = torch.cuda.get_device_name(0).replace(" ", "_").replace('"', "_").replace("\\", "_")
    cache = tmp_path / "tiles.json"
    packed = upd | (16 << 8) | (32 << 16)
    cache.write_text(json.dumps({f"blas/8.8.8.8/kind{kind}/N{N}/{dev}": packed}))
    s, fat, lng = gh.make_solver(dims, mass, prec=prec, seed=1025, max_rhs=N)
    s.set_tune_cache(cache)
    b = hi.gaussian_sources(dims, N, seed=2025)
    X, info = s.solve(b, tol=1e-10)
    assert info["status"] == 0
    assert _oracle_rel_res(dims, fat, lng, mass, b, gh.to_np(X)).max() <= 1e-10
    assert f'"blas/8.8.8.8/kind{kind}/N{N}/{dev}": {packed}' in cache.read_text()


@pytest.mark.parametrize("prec,kind", [("mixed_f16", 3), ("mixed_bf16", 4)])
@pytest.mark.parametrize("N", [16, 32])
@pytest.mark.parametrize("dims", [(8, 8, 8, 8), (6, 6, 6, 6)])
def test_tensor_core_blas_converge(tmp_path, prec, kind, N, dims):
    """The tensor-core fused update (bit 24 of the cached BLAS choice), fused
    W + Gram (bit 25) and Gram P^dag AP (bit 26), each alone and all
    together, forced through the
    tuning cache for the 16-bit forms; 6^4 has 3 V_h = 1944 rows, a ragged
    last 16-row tile (8 rows) and a ragged 128-row Gram tile (24 rows).
    Each solve meets tol on the oracle's residual, in about as many
    iterations as with the FP32-pipe kernels."""
    import json
    torch = gh.torch_mod()
    mass = 0.05
    dev = torch.cuda.get_device_name(0).replace(" ", "_").replace('"', "_").replace("\\", "_")
    tag = ".".join(str(d) for d in dims)
    b = hi.gaussian_sources(dims, N, seed=2026)
    iters = {}
    for name, flags in (("pipes", 0), ("upd", 1 << 24), ("wgram", 1 << 25), ("gram", 1 << 26),
                        ("all", (1 << 24) | (1 << 25) | (1 << 26))):
        cache = tmp_path / f"tiles_{name}.json"
        packed = 8 | (16 << 8) | (32 << 16) | flags
        cache.write_text(json.dumps({f"blas/{tag}/kind{kind}/N{N}/{dev}": packed}))
        s, fat, lng = gh.make_solver(dims, mass, prec=prec, seed=1026, max_rhs=N)
        s.set_tune_cache(cache)
        try:
            X, info = s.solve(b, tol=1e-10)
        except Exception as e:  # name the variant that failed
            raise AssertionError(f"{name}: {e}") from e
        assert info["status"] == 0, name
        assert _oracle_rel_res(dims, fat, lng, mass, b, gh.to_np(X)).max() <= 1e-10, name
        iters[name] = info["iters"]
    for name in ("upd", "wgram", "gram", "all"):
        assert abs(iters[name] - iters["pipes"]) <= max(3, iters["pipes"] // 10), iters
