"""Link gradient through the C ABI (blockcg_link_grad) and the differentiable
solve (autograd.HisqSolve) against the CPU oracle's gradient, whose formula
is pinned by finite differences in test_oracle_grad.py."""
import numpy as np
import pytest

import hisq_inputs as hi
from oracle import hisq

from gpu_helpers import ensure_built, make_solver, to_np

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 4, 8), (2, 2, 2, 2)])
@pytest.mark.parametrize("N", [1, 3])
@pytest.mark.parametrize("antiperiodic", [False, True])
def test_link_grad_kernel_matches_oracle(dims, N, antiperiodic):
    """Same X and Lam on both sides: the kernel's outer-product sums equal the
    oracle's to FP64 rounding (each entry sums 2N products of two stencil
    outputs)."""
    s, fat, lng = make_solver(dims, 0.1, prec="f64", seed=1200, max_rhs=4,
                              antiperiodic_t=antiperiodic)
    X = hi.gaussian_sources(dims, N, 1201)
    Lam = hi.gaussian_sources(dims, N, 1202)
    gf, gl = s.link_grad(X, Lam)
    rf, rl = hisq.link_grad(dims, fat, lng, X, Lam, antiperiodic)
    for got, ref in ((gf, rf), (gl, rl)):
        got = to_np(got)
        assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()
    # one output only
    gf2, gl2 = s.link_grad(X, Lam, lng=False)
    assert gl2 is None and np.array_equal(to_np(gf2), to_np(gf))


def test_autograd_quadratic_loss_16x4():
    """L = sum_i phi_i^dag A^-1 phi_i on 16^4, m = 0.05, N = 8 (F64 form to
    1e-12): the loss and its gradients with respect to the fat and long links
    and to phi match the oracle's (oracle CG solution, oracle gradient).
    The error bound: x has relative error <~ kappa * 1e-12 (kappa ~ 1.7e3 at
    m = 0.05), and the gradient is bilinear in x."""
    import torch
    from paper_1710_09745_gb300.autograd import hisq_solve
    ensure_built()
    dims, mass, N = (16, 16, 16, 16), 0.05, 8
    fat, lng = hi.random_links(dims, 1300)
    phi_np = hi.gaussian_sources(dims, N, 1301)
    s, _, _ = make_solver(dims, mass, prec="f64", links=(fat, lng), max_rhs=N)
    f = torch.tensor(fat, device="cuda", requires_grad=True)
    l = torch.tensor(lng, device="cuda", requires_grad=True)
    phi = torch.tensor(phi_np, device="cuda", requires_grad=True)
    x = hisq_solve(f, l, phi, s, tol=1e-12)
    loss = (phi.conj() * x).sum().real
    loss.backward()
    # oracle: CG solution and the gradient formula (self-adjoint: lam = x)
    xo, _, res = hisq.cg(dims, fat, lng, mass, phi_np, tol=1e-12, max_iter=20000)
    assert res.max() <= 1e-12
    rf, rl = hisq.link_grad(dims, fat, lng, xo, xo)
    lo = float(np.real(np.vdot(phi_np.reshape(-1), xo.reshape(-1))))
    assert abs(loss.item() - lo) <= 1e-9 * abs(lo)
    for got, ref in ((f.grad, rf), (l.grad, rl)):
        assert np.abs(to_np(got) - ref).max() <= 1e-7 * np.abs(ref).max()
    # phi enters twice (phi^dag and x = A^-1 phi): dL/dphi = 2 x
    assert np.abs(to_np(phi.grad) - 2 * xo).max() <= 1e-7 * np.abs(xo).max()


def test_autograd_general_loss_adjoint_solve():
    """L = Re sum_i c_i^dag A^-1 phi_i with c independent of phi: the adjoint
    block A^-1 c differs from x, exercising both outer-product terms."""
    import torch
    from paper_1710_09745_gb300.autograd import hisq_solve
    ensure_built()
    dims, mass, N = (8, 8, 8, 8), 0.1, 4
    fat, lng = hi.random_links(dims, 1400)
    phi_np = hi.gaussian_sources(dims, N, 1401)
    c_np = hi.gaussian_sources(dims, N, 1402)
    s, _, _ = make_solver(dims, mass, prec="f64", links=(fat, lng), max_rhs=N)
    f = torch.tensor(fat, device="cuda", requires_grad=True)
    l = torch.tensor(lng, device="cuda", requires_grad=True)
    phi = torch.tensor(phi_np, device="cuda", requires_grad=True)
    c = torch.tensor(c_np, device="cuda")
    x = hisq_solve(f, l, phi, s, tol=1e-12)
    (c.conj() * x).sum().real.backward()
    xo, _, _ = hisq.cg(dims, fat, lng, mass, phi_np, tol=1e-12, max_iter=20000)
    lo, _, _ = hisq.cg(dims, fat, lng, mass, c_np, tol=1e-12, max_iter=20000)
    rf, rl = hisq.link_grad(dims, fat, lng, xo, lo)
    for got, ref in ((f.grad, rf), (l.grad, rl)):
        assert np.abs(to_np(got) - ref).max() <= 1e-8 * np.abs(ref).max()
    assert np.abs(to_np(phi.grad) - lo).max() <= 1e-8 * np.abs(lo).max()


def test_autograd_central_difference_4x4():
    """Central finite difference (h = 1e-6, FP64) of the GPU loss along a
    random direction through all fat links, against the autograd gradient.
    Native-FP64 solves to 1e-13: each loss carries an error up to
    |phi| |A^-1| |r| ~ 100 * 1e-13 * |phi|^2 ~ 2e-8, i.e. ~1e-2 in the quotient,
    against a directional derivative of ~1e3 (bound 1e-5 relative; 1e-4 asserted)."""
    import torch
    from paper_1710_09745_gb300.autograd import hisq_solve
    ensure_built()
    dims, mass, N, h = (4, 4, 4, 4), 0.1, 2, 1e-6
    fat, lng = hi.random_links(dims, 1500)
    phi_np = hi.gaussian_sources(dims, N, 1501)
    s, _, _ = make_solver(dims, mass, prec="f64_native", links=(fat, lng), max_rhs=N)
    phi = torch.tensor(phi_np, device="cuda")
    lt = torch.tensor(lng, device="cuda")

    def loss_of(fv):
        x = hisq_solve(fv, lt, phi, s, tol=1e-13)
        return (phi.conj() * x).sum().real

    f = torch.tensor(fat, device="cuda", requires_grad=True)
    loss_of(f).backward()
    rng = np.random.default_rng(7)
    d = torch.tensor(rng.standard_normal(fat.shape) + 1j * rng.standard_normal(fat.shape),
                     device="cuda")
    with torch.no_grad():
        fd = (loss_of(torch.tensor(fat, device="cuda") + h * d).item() -
              loss_of(torch.tensor(fat, device="cuda") - h * d).item()) / (2 * h)
    pred = float(torch.real(torch.sum(torch.conj(f.grad) * d)).item())
    assert abs(fd - pred) <= 1e-4 * abs(pred), (fd, pred)
