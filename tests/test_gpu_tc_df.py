"""GPU parity of the tensor-core double-float kernels (split bf16 products on
mma.sync): the stencil of Eq. 2 (Sec. 6.2) against the CPU oracle in single halves,
the normal operator, columns of very different magnitude, the fallback for
unsupported widths, whole solves and a full-size sampled check; the fused
block update of Algorithm 1 (Sec. 6.3) through whole solves."""
import numpy as np
import pytest

import hisq_inputs as hi
from oracle import hisq
from tests import gpu_helpers as gh
from tests import lattice_helpers as lh

pytestmark = pytest.mark.gpu

DIMS = (6, 8, 10, 12)   # Vh = 2880: 360 groups of 8 sites over many CTAs
TC = 8192               # blockcg_params.dslash_variant: tensor-core stencil
ASYNC = 512
# the register-tile bits of the variant do not matter for this kernel
TC_VARIANTS = [TC + 1]


@pytest.mark.parametrize("variant", TC_VARIANTS)
@pytest.mark.parametrize("N", [16, 32])
@pytest.mark.parametrize("parity", [0, 1])
def test_dslash_tc_parity(variant, N, parity):
    s, fat, lng = gh.make_solver(DIMS, 0.1, prec="f64", seed=1011, max_rhs=N, dslash_variant=variant)
    psi = hi.gaussian_sources(DIMS, N, seed=99 + N)
    out = gh.to_np(s.dslash(psi, parity))
    ref = hisq.dslash(DIMS, fat, lng, psi, parity)
    assert gh.rel_err(out, ref) < gh.TOL["f64"]


@pytest.mark.parametrize("variant", TC_VARIANTS)
@pytest.mark.parametrize("N", [16, 32])
def test_dslash_tc_column_scales(variant, N):
    """Columns spanning 10^-6 .. 10^6: every column keeps its own relative
    accuracy (one power-of-two scale per right-hand side)."""
    s, fat, lng = gh.make_solver(DIMS, 0.1, prec="f64", seed=1012, max_rhs=N, dslash_variant=variant)
    psi = hi.gaussian_sources(DIMS, N, seed=300 + N)
    psi *= (10.0 ** (np.arange(N) % 13 - 6))[:, None, None]
    out = gh.to_np(s.dslash(psi, 1))
    ref = hisq.dslash(DIMS, fat, lng, psi, 1)
    for j in range(N):
        assert gh.rel_err(out[j], ref[j]) < gh.TOL["f64"], j


def test_dslash_tc_zero_column_and_scaled_links():
    """An all-zero right-hand side, and links scaled by 37 (no longer below 1):
    the per-site link scale follows them."""
    N = 16
    fat, lng = hi.random_links(DIMS, 1013)
    fat, lng = 37.0 * fat, 37.0 * lng
    s, _, _ = gh.make_solver(DIMS, 0.1, prec="f64", links=(fat, lng), max_rhs=N,
                             dslash_variant=TC + 1)
    psi = hi.gaussian_sources(DIMS, N, seed=301)
    psi[5] = 0.0
    out = gh.to_np(s.dslash(psi, 0))
    ref = hisq.dslash(DIMS, fat, lng, psi, 0)
    assert gh.rel_err(out, ref) < gh.TOL["f64"]
    assert np.all(out[5] == 0.0)


@pytest.mark.parametrize("N", [1, 5, 8, 33])
def test_dslash_tc_fallback_widths(N):
    """Widths the tensor-core kernel does not take run the cp.async kernel."""
    s, fat, lng = gh.make_solver(DIMS, 0.1, prec="f64", seed=1014, max_rhs=max(N, 16),
                                 dslash_variant=TC + 1)
    psi = hi.gaussian_sources(DIMS, N, seed=400 + N)
    out = gh.to_np(s.dslash(psi, 1))
    ref = hisq.dslash(DIMS, fat, lng, psi, 1)
    assert gh.rel_err(out, ref) < gh.TOL["f64"]


@pytest.mark.parametrize("variant", TC_VARIANTS)
@pytest.mark.parametrize("N", [16, 32])
def test_apply_MdagM_tc(variant, N):
    s, fat, lng = gh.make_solver(DIMS, 0.1, prec="f64", seed=1015, max_rhs=N, dslash_variant=variant)
    v = hi.gaussian_sources(DIMS, N, seed=500 + N)
    out = gh.to_np(s.apply_MdagM(v))
    ref = hisq.apply_A(DIMS, fat, lng, 0.1, v)
    assert gh.rel_err(out, ref) < gh.TOL["f64"]


def test_apply_tc_antiperiodic_tiny_lattice():
    """4^4 with antiperiodic t: the +-3 hops wrap onto coincident sites."""
    dims = (4, 4, 4, 4)
    N = 16
    s, fat, lng = gh.make_solver(dims, 0.2, prec="f64", seed=1016, max_rhs=N, dslash_variant=TC + 1,
                                 antiperiodic_t=1)
    v = hi.gaussian_sources(dims, N, seed=501)
    out = gh.to_np(s.apply_MdagM(v))
    ref = hisq.apply_A(dims, fat, lng, 0.2, v, antiperiodic_t=True)
    assert gh.rel_err(out, ref) < gh.TOL["f64"]


@pytest.mark.parametrize("variant,N", [(TC + 1, 16), (TC + 1, 32)])
def test_solve_tc_against_oracle(variant, N):
    """Whole block-CGrQ solves with the tensor-core stencil: the true residual
    meets tol, the solution matches the oracle's, and the iteration count
    stays within a few percent of the CUDA-core double-float stencil's."""
    dims = (8, 8, 8, 12)
    mass = 0.05
    b = hi.gaussian_sources(dims, N, seed=2007 + N)
    s, fat, lng = gh.make_solver(dims, mass, prec="f64", seed=1017, max_rhs=N, dslash_variant=variant)
    X, info = s.solve(b, tol=1e-12)
    assert info["status"] == 0, info
    X = gh.to_np(X)
    r = b - hisq.apply_A(dims, fat, lng, mass, X)
    rel = np.linalg.norm(r.reshape(N, -1), axis=1) / np.linalg.norm(b.reshape(N, -1), axis=1)
    assert rel.max() <= 1e-12 * 1.01, rel
    xo = np.stack([hisq.cg(dims, fat, lng, mass, b[j:j + 1], tol=1e-13, max_iter=20000)[0][0]
                   for j in range(0, N, 7)])
    err = np.linalg.norm((X[::7] - xo).reshape(len(xo), -1), axis=1) / \
        np.linalg.norm(xo.reshape(len(xo), -1), axis=1)
    assert err.max() < 1e-8, err
    s2, _, _ = gh.make_solver(dims, mass, prec="f64", links=(fat, lng), max_rhs=N,
                              dslash_variant=ASYNC + 2)
    _, info2 = s2.solve(b, tol=1e-12)
    assert info["iters"] <= 1.05 * info2["iters"] + 2, (info["iters"], info2["iters"])


def test_apply_tc_full_size_sampled():
    """32^4, N = 16 (the benchmark workload) with the tensor-core stencil:
    sampled output sites against the oracle."""
    dims = (32, 32, 32, 32)
    N = 16
    fat, lng = hi.random_links_torch(dims, 1001, "cpu")
    fat, lng = fat.numpy(), lng.numpy()
    b = hi.gaussian_sources(dims, N, 2100)
    s, _, _ = gh.make_solver(dims, 0.01, prec="f64", links=(fat, lng), max_rhs=N,
                             dslash_variant=TC + 1)
    out = gh.to_np(s.apply_MdagM(b))
    rng = np.random.default_rng(9)
    sites = np.sort(rng.choice(lh.even_sites(dims), size=48, replace=False))
    for j in (0, 7, 15):
        ref = hisq.apply_A_sites(dims, fat, lng, 0.01, b[j], sites)
        got = out[j][sites >> 1]
        assert np.abs(got - ref).max() < gh.TOL["f64"] * np.abs(ref).max()


def _oracle_rel_res(dims, fat, lng, mass, b, X):
    r = b - hisq.apply_A(dims, fat, lng, mass, X)
    return np.linalg.norm(r.reshape(len(b), -1), axis=1) / np.linalg.norm(b.reshape(len(b), -1), axis=1)


@pytest.mark.parametrize("dims", [(8, 8, 8, 8), (6, 6, 6, 6)])
@pytest.mark.parametrize("stencil", [ASYNC + 2, TC + 1])
def test_tc_blas_df_converges(tmp_path, dims, stencil):
    """The tensor-core double-float block BLAS as exact split bf16 products:
    the fused update (Q = W S^-1, P = Q + P S^dag, X += P beta C; bit 24 of
    the cached BLAS choice), W = Q - AP beta with the Gram W^dag W (bit 25)
    and the Gram P^dag AP (bit 26), each alone and all together, forced
    through the tuning cache, with the CUDA-core and the tensor-core stencil.
    6^4 has 3 V_h = 1944 rows: a ragged last 16-row tile and a ragged 64-row
    Gram tile (24 rows).  Each solve to 1e-12 meets tol on the oracle's
    residual, the all-tensor-core solve matches the oracle's solution, and
    every variant takes about as many iterations as the CUDA-core kernels."""
    import json
    torch = gh.torch_mod()
    mass, N = 0.05, 16
    dev = torch.cuda.get_device_name(0).replace(" ", "_").replace('"', "_").replace("\\", "_")
    tag = ".".join(str(d) for d in dims)
    b = hi.gaussian_sources(dims, N, seed=2031)
    iters = {}
    for name, flags in (("pipes", 0), ("upd", 1 << 24), ("wgram", 1 << 25), ("gram", 1 << 26),
                        ("all", (1 << 24) | (1 << 25) | (1 << 26))):
        cache = tmp_path / f"tiles_{name}.json"
        packed = 8 | (16 << 8) | (32 << 16) | flags
        cache.write_text(json.dumps({f"blas/{tag}/kind0/N{N}/{dev}": packed}))
        s, fat, lng = gh.make_solver(dims, mass, prec="f64", seed=1031, max_rhs=N,
                                     dslash_variant=stencil)
        s.set_tune_cache(cache)
        X, info = s.solve(b, tol=1e-12)
        assert info["status"] == 0, name
        X = gh.to_np(X)
        assert _oracle_rel_res(dims, fat, lng, mass, b, X).max() <= 1.01e-12, name
        iters[name] = info["iters"]
        if name == "all":
            xo = hisq.cg(dims, fat, lng, mass, b[:2], tol=1e-13, max_iter=20000)[0]
            err = np.linalg.norm((X[:2] - xo).reshape(2, -1), axis=1) / \
                np.linalg.norm(xo.reshape(2, -1), axis=1)
            assert err.max() < 1e-8, err
    for name in ("upd", "wgram", "gram", "all"):
        assert abs(iters[name] - iters["pipes"]) <= max(3, iters["pipes"] // 20), iters


def test_tc_blas_df_width_32(tmp_path):
    """N = 32: the tensor-core W = Q - AP beta with W^dag W (bit 25) and
    P^dag AP (bit 26), alone and together (the fused update stays on the
    CUDA cores at this width; bit 24 falls back to it), with the tensor-core
    stencil: each solve to 1e-12 meets tol on the oracle's residual in about
    as many iterations as the CUDA-core kernels, and the all-tensor-core
    solve matches the oracle's solution."""
    import json
    torch = gh.torch_mod()
    dims, mass, N = (8, 8, 8, 8), 0.05, 32
    dev = torch.cuda.get_device_name(0).replace(" ", "_").replace('"', "_").replace("\\", "_")
    b = hi.gaussian_sources(dims, N, seed=2032)
    iters = {}
    for name, flags in (("pipes", 0), ("wgram", 1 << 25), ("gram", 1 << 26),
                        ("all", (1 << 24) | (1 << 25) | (1 << 26))):
        cache = tmp_path / f"tiles32_{name}.json"
        packed = 8 | (8 << 8) | (16 << 16) | flags
        cache.write_text(json.dumps({f"blas/8.8.8.8/kind0/N{N}/{dev}": packed}))
        s, fat, lng = gh.make_solver(dims, mass, prec="f64", seed=1032, max_rhs=N,
                                     dslash_variant=TC + 1)
        s.set_tune_cache(cache)
        X, info = s.solve(b, tol=1e-12)
        assert info["status"] == 0, name
        X = gh.to_np(X)
        assert _oracle_rel_res(dims, fat, lng, mass, b, X).max() <= 1.01e-12, name
        iters[name] = info["iters"]
        if name == "all":
            xo = hisq.cg(dims, fat, lng, mass, b[:2], tol=1e-13, max_iter=20000)[0]
            err = np.linalg.norm((X[:2] - xo).reshape(2, -1), axis=1) / \
                np.linalg.norm(xo.reshape(2, -1), axis=1)
            assert err.max() < 1e-8, err
    for name in ("wgram", "gram", "all"):
        assert abs(iters[name] - iters["pipes"]) <= max(3, iters["pipes"] // 20), iters
