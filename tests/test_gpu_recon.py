"""Two-row link storage (params.link_recon = 12) for the 32- and 16-bit
forms: the stencil rebuilds the third row of every hop matrix from the first
two.  Parity against the oracle's full-matrix operator at the same tolerance
as the full storage, every plain-kernel tile, both boundary conditions; links
that are not real multiples of SU(3) matrices are refused on load."""
import numpy as np
import pytest

import hisq_inputs as hi
from oracle import hisq

from gpu_helpers import TOL, make_solver, rel_err, to_np

pytestmark = pytest.mark.gpu

PRECS = ["mixed_f32", "mixed_f16", "mixed_bf16"]
DIMS = (4, 4, 4, 8)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("antiperiodic", [False, True])
@pytest.mark.parametrize("N", [1, 4, 6])
def test_recon_operator_parity(prec, antiperiodic, N):
    s, fat, lng = make_solver(DIMS, 0.05, prec=prec, seed=1700, max_rhs=8,
                              antiperiodic_t=antiperiodic, link_recon=12)
    v = hi.gaussian_sources(DIMS, N, 1701)
    for parity in (0, 1):
        out = to_np(s.dslash(v, parity))
        ref = hisq.dslash(DIMS, fat, lng, v, parity, antiperiodic)
        assert rel_err(out, ref) < TOL[prec], parity
    out = to_np(s.apply_MdagM(v))
    ref = hisq.apply_A(DIMS, fat, lng, 0.05, v, antiperiodic)
    assert rel_err(out, ref) < TOL[prec]


@pytest.mark.parametrize("R", [1, 2, 4, 8])
def test_recon_every_tile(R):
    s, fat, lng = make_solver(DIMS, 0.05, prec="mixed_f32", seed=1710, max_rhs=8,
                              dslash_variant=R, link_recon=12)
    v = hi.gaussian_sources(DIMS, 8, 1711)
    out = to_np(s.apply_MdagM(v))
    ref = hisq.apply_A(DIMS, fat, lng, 0.05, v)
    assert rel_err(out, ref) < TOL["mixed_f32"]


def test_recon_unit_links():
    fat, lng = hi.unit_links(DIMS)
    s, _, _ = make_solver(DIMS, 0.1, prec="mixed_f32", links=(fat, lng), max_rhs=2, link_recon=12)
    v = hi.gaussian_sources(DIMS, 2, 1720)
    assert rel_err(to_np(s.apply_MdagM(v)), hisq.apply_A(DIMS, fat, lng, 0.1, v)) < TOL["mixed_f32"]


@pytest.mark.parametrize("damage", ["scaled_link", "general_matrix", "sign_flip"])
def test_recon_refuses_links_outside_scaled_su3(damage):
    from paper_1710_09745_gb300 import BlockCGError
    fat, lng = hi.random_links(DIMS, 1730)
    fat = fat.copy()
    if damage == "scaled_link":      # one link with another scale
        fat[2, 17] *= 1.01
    elif damage == "general_matrix":  # not unitary
        fat[1, 5, 0, 1] += 0.3
    else:                             # -U has determinant -1: not a positive multiple's pattern
        fat[3, 40] *= -1.0
    with pytest.raises(BlockCGError) as e:
        make_solver(DIMS, 0.1, prec="mixed_f32", links=(fat, lng), max_rhs=2, link_recon=12)
    assert e.value.status == 1


@pytest.mark.parametrize("prec", ["mixed_f32", "mixed_f16"])
def test_recon_solve_reaches_tolerance(prec):
    dims, mass = (8, 8, 8, 8), 0.05
    s, fat, lng = make_solver(dims, mass, prec=prec, seed=1740, max_rhs=4, link_recon=12)
    b = hi.gaussian_sources(dims, 4, 1741)
    X, info = s.solve(b, tol=1e-10)
    assert info["status"] == 0, info
    r = b - hisq.apply_A(dims, fat, lng, mass, to_np(X))
    rel = np.linalg.norm(r.reshape(4, -1), axis=1) / np.linalg.norm(b.reshape(4, -1), axis=1)
    assert rel.max() <= 1.05e-10
    # the CG baseline uses the same links
    Xc, ic = s.solve_cg(b[:1], tol=1e-10)
    assert ic["status"] == 0, ic
