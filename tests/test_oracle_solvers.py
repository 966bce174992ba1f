"""Pins of the oracle's CG and of the NumPy blockCGrQ / thin-QR / reliable
update transcription (Algorithms 1-3) against dense linear algebra and the
algebraic invariants of the method."""
import numpy as np
import pytest

import hisq_inputs as hi
from oracle import block, dense, hisq


def _setup(dims, mass, n, seed=0):
    fat, lng = hi.random_links(dims, seed=100 + seed)
    b = hi.gaussian_sources(dims, n, seed=200 + seed)
    return fat, lng, b


@pytest.mark.parametrize("dims,mass", [((2, 2, 2, 2), 0.1), ((4, 4, 4, 4), 0.1)])
def test_cg_matches_dense_solve(dims, mass):
    fat, lng, b = _setup(dims, mass, 3)
    A = dense.dense_A(dims, fat, lng, mass)
    x, iters, res = hisq.cg(dims, fat, lng, mass, b, tol=1e-13)
    B = block.as_columns(b)
    Xd = np.linalg.solve(A, B)
    X = block.as_columns(x)
    rel = np.linalg.norm(X - Xd, axis=0) / np.linalg.norm(Xd, axis=0)
    assert rel.max() < 1e-10, rel
    assert res.max() <= 1e-13
    # reported true residual agrees with a dense recomputation
    r = np.linalg.norm(B - A @ X, axis=0) / np.linalg.norm(B, axis=0)
    assert np.allclose(r, res, rtol=1e-3, atol=1e-14)


def test_cg_iterates_are_krylov_optimal():
    """x_k of CG minimises the A-norm error over K_k(A, b) (Galerkin condition):
    compare with the dense projected solve on an orthonormal Krylov basis."""
    dims = (4, 4, 4, 4)
    mass = 0.2
    fat, lng, b = _setup(dims, mass, 1, seed=3)
    A = dense.dense_A(dims, fat, lng, mass)
    bv = b[0].ravel()
    for k in (1, 2, 5, 9):
        K = np.empty((bv.size, k), dtype=np.complex128)
        v = bv.copy()
        for j in range(k):
            K[:, j] = v
            v = A @ v
        Qk, _ = np.linalg.qr(K)
        y = np.linalg.solve(Qk.conj().T @ A @ Qk, Qk.conj().T @ bv)
        x_opt = Qk @ y
        xk = hisq.cg_iterates(dims, fat, lng, mass, b[0], k).ravel()
        assert np.linalg.norm(xk - x_opt) < 1e-9 * np.linalg.norm(x_opt), k


def test_block_cdot_bruteforce():
    rng = np.random.default_rng(1)
    X = rng.standard_normal((7, 3)) + 1j * rng.standard_normal((7, 3))
    Y = rng.standard_normal((7, 4)) + 1j * rng.standard_normal((7, 4))
    K = block.block_cdot(X, Y)
    for i in range(3):
        for j in range(4):
            s = 0j
            for k in range(7):
                s += complex(X[k, i]).conjugate() * complex(Y[k, j])
            assert abs(K[i, j] - s) < 1e-13
    a = rng.standard_normal((3, 4)) + 1j * rng.standard_normal((3, 4))
    Z = block.block_caxpy(Y, X, a)
    for k in range(7):
        for j in range(4):
            s = complex(Y[k, j])
            for i in range(3):
                s += complex(X[k, i]) * complex(a[i, j])
            assert abs(Z[k, j] - s) < 1e-13


def test_thin_qr_against_householder():
    rng = np.random.default_rng(2)
    M = rng.standard_normal((200, 6)) + 1j * rng.standard_normal((200, 6))
    Q, R = block.thin_qr(M)
    assert np.abs(Q.conj().T @ Q - np.eye(6)).max() < 1e-12
    assert np.abs(Q @ R - M).max() < 1e-12
    assert np.abs(np.tril(R, -1)).max() == 0
    assert np.all(np.abs(np.diag(R).imag) < 1e-14) and np.all(np.diag(R).real > 0)
    # Householder QR is unique up to a diagonal unitary: |R| agrees
    Qh, Rh = np.linalg.qr(M)
    assert np.abs(np.abs(R) - np.abs(Rh)).max() < 1e-10


def test_block_cg_rq_n1_equals_cg_iterates():
    """For N=1 blockCGrQ reduces to CG (Sec. 4): same iterates."""
    dims = (4, 4, 4, 4)
    mass = 0.1
    fat, lng, b = _setup(dims, mass, 1, seed=4)
    A = lambda P: block.as_columns(hisq.apply_A(dims, fat, lng, mass,  # noqa: E731
                                                block.from_columns(P, 128)))
    hist = []
    block.block_cg_rq(A, block.as_columns(b), tol=1e-30, max_iter=30, history=hist)
    for k in (1, 5, 12, 30):
        xk = hisq.cg_iterates(dims, fat, lng, mass, b[0], k).ravel()
        xb = hist[k - 1]["X"][:, 0]
        assert np.linalg.norm(xb - xk) < 1e-10 * np.linalg.norm(xk), k


def test_block_cg_rq_invariants_and_solution():
    dims = (4, 4, 4, 4)
    mass = 0.1
    N = 4
    fat, lng, b = _setup(dims, mass, N, seed=5)
    Ad = dense.dense_A(dims, fat, lng, mass)
    A = lambda P: Ad @ P  # noqa: E731
    B = block.as_columns(b)
    hist = []
    X, info = block.block_cg_rq(A, B, tol=1e-12, history=hist)
    Xd = np.linalg.solve(Ad, B)
    assert np.abs(X - Xd).max() < 1e-9 * np.abs(Xd).max()
    assert info["true_rel_res"].max() <= 1e-12
    Xprev = np.zeros_like(B)
    for k, h in enumerate(hist[:40]):
        assert np.abs(h["QtQ"] - np.eye(N)).max() < 1e-10          # Q^dag Q = I
        assert np.abs(h["QtP"] - np.eye(N)).max() < 1e-9           # Q_old^dag P = I
        assert np.abs(h["PAP"] - h["PAP"].conj().T).max() < 1e-10 * np.abs(h["PAP"]).max()
        assert np.linalg.eigvalsh(h["PAP"]).min() > 0
        # |R_i|^2 = sum_j |C_ji|^2 against the true residual of the iterate
        true = np.linalg.norm(B - Ad @ h["X"], axis=0)
        assert np.allclose(block.column_norms(h["C"]), true, rtol=1e-8)
        Xprev = h["X"]


def test_block_cg_rq_fewer_iterations_than_cg():
    dims = (4, 4, 4, 4)
    mass = 0.1
    N = 8
    fat, lng, b = _setup(dims, mass, N, seed=6)
    Ad = dense.dense_A(dims, fat, lng, mass)
    _, info = block.block_cg_rq(lambda P: Ad @ P, block.as_columns(b), tol=1e-10)
    _, iters, _ = hisq.cg(dims, fat, lng, mass, b, tol=1e-10)
    assert info["iterations"] < iters.max()


def test_block_cg_rq_finite_termination_tiny():
    """Exact arithmetic ends in at most L/N iterations (Sec. 4); L = 24 on 2^4."""
    dims = (2, 2, 2, 2)
    mass = 0.1
    N = 4
    fat, lng, b = _setup(dims, mass, N, seed=7)
    Ad = dense.dense_A(dims, fat, lng, mass)
    X, info = block.block_cg_rq(lambda P: Ad @ P, block.as_columns(b), tol=1e-11)
    assert info["iterations"] <= 24 // N + 2
    Xd = np.linalg.solve(Ad, block.as_columns(b))
    assert np.abs(X - Xd).max() < 1e-9 * np.abs(Xd).max()


def test_reliable_updates_mixed_precision():
    """Algorithm 3 with P, Q, AP rounded to complex64: converges to 1e-10 in the
    true residual, keeps Q_old^dag P = I across updates, and needs about as many
    iterations as the FP64 solve (a wrong S = C C_old^-1 loses the Krylov space
    at every update and multiplies the iteration count)."""
    dims = (4, 4, 4, 4)
    mass = 0.1
    N = 4
    fat, lng, b = _setup(dims, mass, N, seed=8)
    Ad = dense.dense_A(dims, fat, lng, mass)
    sloppy = lambda a: a.astype(np.complex64).astype(np.complex128)  # noqa: E731
    A_s = lambda P: sloppy(Ad @ sloppy(P))  # noqa: E731
    B = block.as_columns(b)
    _, info64 = block.block_cg_rq(lambda P: Ad @ P, B, tol=1e-10)
    for delta in (0.5, 0.1, 0.01):
        hist = []
        X, info = block.block_cg_rq(lambda P: Ad @ P, B, tol=1e-10, apply_A_sloppy=A_s,
                                    sloppy=sloppy, delta=delta, history=hist)
        assert info["true_rel_res"].max() <= 1e-10
        assert info["reliable_updates"] >= 3
        assert info["iterations"] <= 1.5 * info64["iterations"], (delta, info["iterations"])
        for h in hist:
            assert np.abs(h["QtP"] - np.eye(N)).max() < 1e-3
    # without reliable updates the sloppy solve stalls well above 1e-10
    X2, info2 = block.block_cg_rq(lambda P: A_s(P), B, tol=1e-10, apply_A_sloppy=A_s,
                                  sloppy=sloppy, delta=None, max_iter=400)
    r2 = np.linalg.norm(B - Ad @ X2, axis=0) / np.linalg.norm(B, axis=0)
    assert r2.max() > 1e-9
