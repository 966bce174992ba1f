"""Block-Krylov algebra of the paper in plain NumPy FP64, step by step.

Test infrastructure; see oracle/__init__.py.

Block vectors here are NumPy arrays of shape (L, N): column j is right-hand
side j, L = 3 * (V/2) complex rows (the paper's X^{L x N}).  `as_columns` and
`from_columns` convert from and to the [N][V/2][3] spinor-block layout.

Functions follow, in order and notation:
  block_cdot     K = X^dag Y,  k_ij = sum_k conj(x_ki) y_kj            (Sec. 6.4)
  block_caxpy    Y + X a,      y_kj += sum_i x_ki a_ij                  (Sec. 6.3)
  thin_qr        H = M^dag M; R^dag R = H (Cholesky); Q = M R^-1        (Algorithm 2)
  block_cg_rq    Algorithm 1, with the block reliable update of
                 Algorithm 3 (Y += X; X = 0; R = B - A Y; Q C = R;
                 S = C C_old^-1)
The iterated residual of column i is |R_i|^2 = sum_j |C_ji|^2, the norm of
column i of C, because R = Q C with Q^dag Q = I (the paper prints the index
pair transposed; the column form is the one that follows from R = QC).
"""
from __future__ import annotations

import numpy as np


def as_columns(block: np.ndarray) -> np.ndarray:
    """[N][V/2][3] -> (L, N)."""
    n = block.shape[0]
    return np.ascontiguousarray(block.reshape(n, -1).T)


def from_columns(cols: np.ndarray, vh: int) -> np.ndarray:
    """(L, N) -> [N][V/2][3]."""
    return np.ascontiguousarray(cols.T.reshape(cols.shape[1], vh, 3))


def block_cdot(X: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """K = X^dag Y (block cDotProduct, Sec. 6.4)."""
    return X.conj().T @ Y


def block_caxpy(Y: np.ndarray, X: np.ndarray, a: np.ndarray) -> np.ndarray:
    """Y + X a (block caxpy, Sec. 6.3)."""
    return Y + X @ a


def cholesky_upper(H: np.ndarray) -> np.ndarray:
    """Upper-triangular R with R^dag R = H (H Hermitian positive definite)."""
    Lo = np.linalg.cholesky(H)
    return Lo.conj().T


def thin_qr(M: np.ndarray):
    """Algorithm 2: returns (Q, R) with Q R = M, R upper triangular."""
    H = block_cdot(M, M)
    R = cholesky_upper(H)
    Q = M @ np.linalg.inv(R)
    return Q, R


def column_norms(C: np.ndarray) -> np.ndarray:
    """|R_i| = sqrt(sum_j |C_ji|^2)."""
    return np.sqrt(np.sum(np.abs(C) ** 2, axis=0))


def block_cg_rq(apply_A, B: np.ndarray, tol: float, max_iter: int = 10000, X0=None,
                apply_A_sloppy=None, sloppy=None, delta: float | None = None,
                ru_every: int = 0, history: list | None = None):
    """blockCGrQ (Algorithm 1) with block reliable updates (Algorithm 3).

    apply_A(P) applies the operator to an (L, N) block in full precision;
    apply_A_sloppy / sloppy (a rounding function for stored block vectors)
    model a mixed-precision solve in which P, Q and AP are kept in lower
    precision.  X, the iterated solution update since the last reliable
    update, and Y, the persistent solution accumulator, are full precision.

    A reliable update happens when the maximum relative iterated residual has
    dropped by the factor delta since the last one (delta=None: never), every
    ru_every iterations (0: never), and whenever the iterated residual claims
    convergence but the true residual of Y + X does not.

    Reading of Algorithm 3: C_old is the C in force before the last
    "C = S C" of Algorithm 1, so that S = C C_old^-1 has the same meaning as
    the S of the ordinary iteration (new C times old C inverse).  With the
    true residual equal to the iterated one this gives back that S exactly.

    Returns (solution, info) where info has iterations, reliable_updates and
    the true relative residual per column.
    """
    if apply_A_sloppy is None:
        apply_A_sloppy = apply_A
    if sloppy is None:
        sloppy = lambda a: a  # noqa: E731
    L, N = B.shape
    bnorm = column_norms(B)
    Y = np.zeros_like(B) if X0 is None else np.array(X0, dtype=np.complex128)
    # R = B - A X ; Q C = R ; S = I ; P = 0
    R = B - apply_A(Y)
    Q, C = thin_qr(R)
    Q = sloppy(Q)
    S = np.eye(N, dtype=np.complex128)
    P = np.zeros_like(B)
    X = np.zeros_like(B)
    C_prev = C
    res = column_norms(C) / bnorm
    res_at_ru = res.max()
    it = 0
    n_ru = 0

    def reliable_update():
        nonlocal Y, X, Q, C, S, res, res_at_ru, n_ru
        Y = Y + X
        X = np.zeros_like(B)
        Rt = B - apply_A(Y)
        Qh, C = thin_qr(Rt)
        Q = sloppy(Qh)
        S = C @ np.linalg.inv(C_prev)                        # S = C C_old^-1
        res = column_norms(C) / bnorm
        res_at_ru = res.max()
        n_ru += 1

    while True:
        if res.max() <= tol:
            true = column_norms(B - apply_A(Y + X)) / bnorm
            if true.max() <= tol:
                break
            reliable_update()
            if res.max() <= tol:
                break
        if it >= max_iter:
            break
        P = sloppy(Q + P @ S.conj().T)                       # P = Q + P S^dag
        if history is not None:
            QtP = Q.conj().T @ P
        AP = sloppy(apply_A_sloppy(P))
        PAP = block_cdot(P, AP)
        beta = np.linalg.inv(PAP)                            # beta = (P^dag A P)^-1
        X = X + P @ (beta @ C)                               # X = X + P beta C
        Qn, S = thin_qr(Q - AP @ beta)                       # Q S = Q - A P beta
        Q = sloppy(Qn)
        C_prev = C
        C = S @ C                                            # C = S C
        it += 1
        res = column_norms(C) / bnorm
        if history is not None:
            history.append({"C": C.copy(), "S": S.copy(), "beta": beta.copy(), "PAP": PAP,
                            "QtP": QtP, "QtQ": Q.conj().T @ Q, "X": Y + X})
        if (delta is not None and res.max() < delta * res_at_ru) or \
                (ru_every and it % ru_every == 0):
            reliable_update()
    Y = Y + X
    true = column_norms(B - apply_A(Y)) / bnorm
    return Y, {"iterations": it, "reliable_updates": n_ru, "true_rel_res": true}
