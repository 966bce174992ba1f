"""GPU parity of the tensor-core stencil of the 16-bit forms (FP16 with its
2^4 factor, bfloat16): the stored values are exact mma.sync operands, FP32
accumulation (Sec. 6.2 stencil of Eq. 2).  Single halves and the normal
operator against the CPU oracle at the 16-bit tolerances, the fallback for
other widths and two-row links, and whole mixed-precision solves."""
import numpy as np
import pytest

import hisq_inputs as hi
from oracle import hisq
from tests import gpu_helpers as gh

pytestmark = pytest.mark.gpu

DIMS = (6, 8, 10, 12)
TC = 8192 + 1
PRECS16 = ["mixed_f16", "mixed_bf16"]


def _psi(n, seed):
    # inputs at the magnitude of the solver's normalised block vectors
    return hi.gaussian_sources(DIMS, n, seed=seed) / np.sqrt(3 * np.prod(DIMS) // 2)


@pytest.mark.parametrize("prec", PRECS16)
@pytest.mark.parametrize("N,parity", [(16, 0), (16, 1), (32, 0), (32, 1), (8, 1), (3, 0)])
def test_dslash_tc16_parity(prec, N, parity):
    s, fat, lng = gh.make_solver(DIMS, 0.1, prec=prec, seed=1041, max_rhs=max(N, 16),
                                 dslash_variant=TC)
    psi = _psi(N, 140 + N)
    out = gh.to_np(s.dslash(psi, parity))
    ref = hisq.dslash(DIMS, fat, lng, psi, parity)
    assert gh.rel_err(out, ref) < gh.TOL[prec]


@pytest.mark.parametrize("prec", PRECS16)
@pytest.mark.parametrize("N", [16, 32])
def test_apply_tc16(prec, N):
    s, fat, lng = gh.make_solver(DIMS, 0.1, prec=prec, seed=1042, max_rhs=N, dslash_variant=TC)
    v = _psi(N, 150 + N)
    out = gh.to_np(s.apply_MdagM(v))
    ref = hisq.apply_A(DIMS, fat, lng, 0.1, v)
    assert gh.rel_err(out, ref) < gh.TOL[prec]


def test_tc16_two_row_links_fall_back():
    """Two-row links are not taken by the tensor-core kernel: the plain kernel
    runs and the result still matches."""
    s, fat, lng = gh.make_solver(DIMS, 0.1, prec="mixed_f16", seed=1043, max_rhs=16,
                                 dslash_variant=TC, link_recon=12)
    psi = _psi(16, 160)
    out = gh.to_np(s.dslash(psi, 1))
    ref = hisq.dslash(DIMS, fat, lng, psi, 1)
    assert gh.rel_err(out, ref) < gh.TOL["mixed_f16"]


@pytest.mark.parametrize("prec", PRECS16)
@pytest.mark.parametrize("N", [16, 32])
def test_solve_tc16(prec, N):
    """Mixed-precision block solves with the tensor-core 16-bit stencil meet
    tol on the oracle's residual, in about as many iterations as with the
    CUDA-core stencil."""
    dims, mass = (8, 8, 8, 8), 0.05
    b = hi.gaussian_sources(dims, N, seed=2041 + N)
    iters = {}
    for name, v in (("tc", TC), ("plain", 4)):
        s, fat, lng = gh.make_solver(dims, mass, prec=prec, seed=1044, max_rhs=N, dslash_variant=v)
        X, info = s.solve(b, tol=1e-10)
        assert info["status"] == 0, name
        r = b - hisq.apply_A(dims, fat, lng, mass, gh.to_np(X))
        rel = np.linalg.norm(r.reshape(N, -1), axis=1) / np.linalg.norm(b.reshape(N, -1), axis=1)
        assert rel.max() <= 1e-10, (name, rel.max())
        iters[name] = info["iters"]
    assert iters["tc"] <= 1.1 * iters["plain"] + 5, iters
