"""CPU FP64 oracle of CholeskyQR2 (Hutter & Solomonik, "Communication-avoiding
CholeskyQR2 for rectangular matrices", arXiv 1710.08471).

TEST INFRASTRUCTURE ONLY. Only the test-suite, the package smoke check and the
CPU-baseline leg of the benchmark may import this module. The GPU library never
calls it and shares no code with it.

The oracle follows the paper's algorithms step by step, in the paper's order
and notation, with numpy FP64 (IEEE round-to-nearest) arithmetic:

* Syrk    (Section II-A):  W = A^T A.
* CholInv (Algorithm 1, Section II-D): [L, Y] = CholInv(W), W = L L^T, Y = L^-1,
  by halving recursion down to dimension 1.
* CQR     (Algorithm CQR, Section II-E): W = Syrk(A); R^T, R^-T = CholInv(W);
  Q = A R^-1.
* CQR2    (Algorithm CQR2, Section II-E): (Q1, R1) = CQR(A); (Q, R2) = CQR(Q1);
  R = R2 R1.
* Panels (the subpanel variant Section V names as future work): CQR2 of each
  column panel after two block projections against the earlier panels
  (panel_cqr2).
* Inverse depth (Section III-A's triangular inverted blocks, the InverseDepth
  parameter of Section IV): CholInv forms the inverse only for the diagonal
  blocks below the top `depth` halvings; L21 and Q come from block forward
  substitution (right_solve).

Readings of points the paper leaves open (each also listed in the design notes):

* Split point of an odd dimension: n1 = floor(n/2) (the paper says "n/2").
* Y21 association: U = L21 Y11 first, then Y21 = -Y22 U, the order of
  Algorithm CFR3D.
* Which Syrk triangle: the upper triangle is kept and mirrored, so W is
  exactly symmetric; CholInv reads only its lower triangle and diagonal.
* Breakdown: a pivot that is not > 0 (or not finite) raises NotSPD with its
  index; the paper states accuracy only for kappa(A) = O(eps^-1/2) and gives
  no recovery.
* Least squares (the paper names least squares as the use, Section I, but
  gives no method): x solves R x = Q^T b by back substitution.

Matrix products use numpy's matmul (a library primitive); nothing is blocked,
fused or reordered beyond what the algorithms state.
"""
from __future__ import annotations

import math

import numpy as np


class NotSPD(ArithmeticError):
    """Cholesky breakdown: pivot `pivot` (0-based, within the CholInv call)
    was not a finite positive number."""

    def __init__(self, pivot: int, value: float):
        super().__init__(f"non-positive or non-finite pivot {value!r} at index {pivot}")
        self.pivot = pivot
        self.value = value


def syrk(A: np.ndarray) -> np.ndarray:
    """W = A^T A (Syrk, Section II-A; Algorithm CQR step 1).

    The upper triangle is computed by a matmul and mirrored into the lower one.
    """
    A = np.asarray(A, dtype=np.float64)
    W = A.T @ A
    U = np.triu(W)
    return U + np.triu(U, 1).T


def _cholinv(A: np.ndarray, offset: int) -> tuple[np.ndarray, np.ndarray]:
    n = A.shape[0]
    if n == 1:
        # Base case of Algorithm 1: L = Chol(A) = sqrt(a), Y = L^-1.
        a = float(A[0, 0])
        if not (a > 0.0) or not math.isfinite(a):
            raise NotSPD(offset, a)
        l = math.sqrt(a)
        return np.array([[l]]), np.array([[1.0 / l]])
    n1 = n // 2
    A11 = A[:n1, :n1]
    A21 = A[n1:, :n1]
    A22 = A[n1:, n1:]
    # Algorithm 1: [L11, Y11] = CholInv(A11)
    L11, Y11 = _cholinv(A11, offset)
    # L21 = A21 Y11^T  (= A21 L11^-T)
    L21 = A21 @ Y11.T
    # [L22, Y22] = CholInv(A22 - L21 L21^T)
    L22, Y22 = _cholinv(A22 - L21 @ L21.T, offset + n1)
    # Y21 = -Y22 L21 Y11, associated as U = L21 Y11, Y21 = -Y22 U (Algorithm CFR3D)
    U = L21 @ Y11
    Y21 = -(Y22 @ U)
    L = np.zeros((n, n))
    Y = np.zeros((n, n))
    L[:n1, :n1] = L11
    L[n1:, :n1] = L21
    L[n1:, n1:] = L22
    Y[:n1, :n1] = Y11
    Y[n1:, :n1] = Y21
    Y[n1:, n1:] = Y22
    return L, Y


def cholinv(W: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """[L, Y] = CholInv(W) (Algorithm 1, Section II-D).

    W symmetric positive definite n x n. Returns lower-triangular L with
    W = L L^T and Y = L^-1 (lower triangular). Raises NotSPD on breakdown.
    """
    W = np.asarray(W, dtype=np.float64)
    if W.ndim != 2 or W.shape[0] != W.shape[1] or W.shape[0] < 1:
        raise ValueError("CholInv needs a non-empty square matrix")
    return _cholinv(W, 0)


def right_solve(B: np.ndarray, L: np.ndarray, Y: np.ndarray, depth: int) -> np.ndarray:
    """X = B L^-T for lower-triangular L whose inverse is known only on the
    diagonal blocks of a depth-`depth` halving (Section III-A's alternative to
    the full inverse: triangular inverted blocks, then Q by multiplications).

    With L = [[L11, 0], [L21, L22]] the two block columns of X L^T = B give
    X1 = B1 L11^-T and X2 = (B2 - X1 L21^T) L22^-T (block forward
    substitution); at depth 0 Y is the full inverse and X = B Y^T.
    """
    n = L.shape[0]
    if depth == 0 or n == 1:
        return B @ Y.T
    n1 = n // 2
    X1 = right_solve(B[:, :n1], L[:n1, :n1], Y[:n1, :n1], depth - 1)
    X2 = right_solve(B[:, n1:] - X1 @ L[n1:, :n1].T, L[n1:, n1:], Y[n1:, n1:], depth - 1)
    return np.hstack([X1, X2])


def _cholinv_depth(A: np.ndarray, offset: int, depth: int) -> tuple[np.ndarray, np.ndarray]:
    # Algorithm 1 whose top `depth` recursion levels do not form Y21: the
    # triangular inverse is computed only below that level (InverseDepth,
    # Section IV), and L21 = A21 L11^-T comes from the block solve instead.
    n = A.shape[0]
    if depth == 0 or n == 1:
        return _cholinv(A, offset)
    n1 = n // 2
    L11, Y11 = _cholinv_depth(A[:n1, :n1], offset, depth - 1)
    L21 = right_solve(A[n1:, :n1], L11, Y11, depth - 1)
    L22, Y22 = _cholinv_depth(A[n1:, n1:] - L21 @ L21.T, offset + n1, depth - 1)
    L = np.zeros((n, n))
    Y = np.zeros((n, n))  # Y21 is not formed
    L[:n1, :n1] = L11
    L[n1:, :n1] = L21
    L[n1:, n1:] = L22
    Y[:n1, :n1] = Y11
    Y[n1:, n1:] = Y22
    return L, Y


def cholinv_depth(W: np.ndarray, depth: int) -> tuple[np.ndarray, np.ndarray]:
    """[L, Y] of Algorithm 1 with inverse depth `depth`: L as before, Y holding
    the inverses of L's diagonal blocks of the depth-`depth` halving only."""
    W = np.asarray(W, dtype=np.float64)
    if W.ndim != 2 or W.shape[0] != W.shape[1] or W.shape[0] < 1 or depth < 0:
        raise ValueError("CholInv needs a non-empty square matrix and depth >= 0")
    return _cholinv_depth(W, 0, depth)


def cqr(A: np.ndarray, inverse_depth: int = 0) -> tuple[np.ndarray, np.ndarray, dict]:
    """[Q, R] = CQR(A) (Algorithm CQR, Section II-E).

    Returns Q, R and the intermediates {W, L, Y, Rinv}. R = L^T is upper
    triangular and Rinv = Y^T = R^-1; Q = A R^-1. With inverse_depth = d > 0
    the inverse is formed only for the diagonal blocks of a depth-d halving
    (cholinv_depth) and Q comes from right_solve; Rinv is then not returned.
    """
    A = np.asarray(A, dtype=np.float64)
    W = syrk(A)  # W = Syrk(A)
    if inverse_depth:
        L, Y = cholinv_depth(W, inverse_depth)
        Q = right_solve(A, L, Y, inverse_depth)  # Q = A R^-1 by block forward substitution
        return Q, np.ascontiguousarray(L.T), dict(W=W, L=L, Y=Y)
    L, Y = cholinv(W)  # R^T, R^-T = CholInv(W)
    R = np.ascontiguousarray(L.T)
    Rinv = np.ascontiguousarray(Y.T)
    Q = A @ Rinv  # Q = MM(A, R^-1)
    return Q, R, dict(W=W, L=L, Y=Y, Rinv=Rinv)


class PassFailed(NotSPD):
    """NotSPD raised inside pass `pass_no` (1 or 2) of CQR2."""

    def __init__(self, pass_no: int, err: NotSPD):
        super().__init__(err.pivot, err.value)
        self.pass_no = pass_no


def cqr2(A: np.ndarray, keep: bool = False, inverse_depth: int = 0):
    """[Q, R] = CQR2(A) (Algorithm CQR2, Section II-E).

    (Q1, R1) = CQR(A); (Q, R2) = CQR(Q1); R = R2 R1. With keep=True also
    returns a dict of intermediates (pass-1 and pass-2 W, L, Y, Rinv, Q1, R1,
    R2). inverse_depth is passed to both CQR passes.
    """
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    if m < n or n < 1:
        raise ValueError("CQR2 needs an m x n matrix with m >= n >= 1")
    try:
        Q1, R1, i1 = cqr(A, inverse_depth)
    except NotSPD as e:
        raise PassFailed(1, e) from None
    try:
        Q, R2, i2 = cqr(Q1, inverse_depth)
    except NotSPD as e:
        raise PassFailed(2, e) from None
    R = np.triu(R2 @ R1)  # R = MM(R2, R1): a product of upper triangles is upper
    if not keep:
        return Q, R
    info = dict(Q1=Q1, R1=R1, R2=R2)
    for k, v in i1.items():
        info[k + "1"] = v
    for k, v in i2.items():
        info[k + "2"] = v
    return Q, R, info


def panel_cqr2(A: np.ndarray, b: int, keep: bool = False):
    """CholeskyQR2 on column panels of width b: the reading of the paper's
    future-work variant that operates on subpanels (Section V, Conclusion).

    Left to right, panel k (columns c0 .. c0 + b - 1) is projected twice
    against the finished panels Q_<k -- C = Q_<k^T V, V = V - Q_<k C; the
    second pass reorthogonalises, as block Gram-Schmidt needs -- and then
    factored by CQR2 (Algorithm CQR2): V = Q_k R_kk. R's block above the
    diagonal block is the sum of the two projections' coefficients. With
    b >= n this is CQR2 itself. Raises PassFailed with the pivot as a column
    index of A when a panel's CholeskyQR2 breaks down.
    """
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    if m < n or n < 1 or b < 1:
        raise ValueError("panel CQR2 needs m >= n >= 1 and b >= 1")
    Q = np.zeros((m, n))
    R = np.zeros((n, n))
    coeffs = []
    for c0 in range(0, n, b):
        c1 = min(n, c0 + b)
        V = A[:, c0:c1].copy()
        if c0:
            Qp = Q[:, :c0]
            for _ in range(2):  # projection, then reorthogonalisation
                C = Qp.T @ V
                V = V - Qp @ C
                R[:c0, c0:c1] += C
                coeffs.append(C)
        try:
            Qk, Rk = cqr2(V)
        except PassFailed as e:
            err = PassFailed(e.pass_no, NotSPD(e.pivot + c0, e.value))
            raise err from None
        Q[:, c0:c1] = Qk
        R[c0:c1, c0:c1] = Rk
    if keep:
        return Q, R, dict(coeffs=coeffs)
    return Q, R


UNIT_ROUNDOFF = 2.0 ** -53


def shift_of(W: np.ndarray, m: int) -> float:
    """Shift of the shifted CholeskyQR pass: s = 11 (m n + n (n+1)) u ||A||_F^2
    with ||A||_F^2 = trace(W) (the published choice for the unconditionally
    stable variant the paper cites in Section I and names as future work in
    Section V; ||A||_2^2 <= ||A||_F^2 keeps it a safe upper bound)."""
    n = W.shape[0]
    return 11.0 * (m * n + n * (n + 1)) * UNIT_ROUNDOFF * float(np.trace(W))


def shifted_cqr(A: np.ndarray) -> tuple[np.ndarray, np.ndarray, dict]:
    """One shifted CholeskyQR pass: W = A^T A + s I, [L, Y] = CholInv(W),
    R = L^T, Q = A R^-1. Q is not orthonormal but well conditioned, which is
    what the following CholeskyQR2 needs."""
    A = np.asarray(A, dtype=np.float64)
    W = syrk(A)
    s = shift_of(W, A.shape[0])
    Ws = W + s * np.eye(W.shape[0])
    L, Y = cholinv(Ws)
    R = np.ascontiguousarray(L.T)
    Q = A @ np.ascontiguousarray(Y.T)
    return Q, R, dict(W=W, shift=s)


def scqr3(A: np.ndarray, keep: bool = False):
    """Shifted CholeskyQR3: (Q0, R0) = shifted CQR(A); (Q, R') = CQR2(Q0);
    R = R' R0."""
    A = np.asarray(A, dtype=np.float64)
    m, n = A.shape
    if m < n or n < 1:
        raise ValueError("sCQR3 needs an m x n matrix with m >= n >= 1")
    try:
        Q0, R0, i0 = shifted_cqr(A)
    except NotSPD as e:
        raise PassFailed(1, e) from None
    try:
        Q, Rp = cqr2(Q0)
    except PassFailed as e:
        raise PassFailed(e.pass_no + 1, e) from None
    R = np.triu(Rp @ R0)
    if keep:
        return Q, R, dict(Q0=Q0, R0=R0, Rp=Rp, **i0)
    return Q, R


def back_substitution(R: np.ndarray, c: np.ndarray) -> np.ndarray:
    """Solve R x = c for upper-triangular R, last unknown first."""
    n = R.shape[0]
    x = np.array(c, dtype=np.float64, copy=True)
    for j in range(n - 1, -1, -1):
        x[j] = x[j] / R[j, j]
        x[:j] -= R[:j, j] * x[j]
    return x


def lstsq(A: np.ndarray, b: np.ndarray, keep: bool = False):
    """Least squares min ||A x - b|| through CQR2: x solves R x = Q^T b."""
    Q, R = cqr2(A)
    c = Q.T @ np.asarray(b, dtype=np.float64)
    x = back_substitution(R, c)
    if keep:
        return x, Q, R
    return x


# ---------------------------------------------------------------- error norms

def orthogonality(Q: np.ndarray) -> float:
    """||Q^T Q - I||_F."""
    G = Q.T @ Q
    G[np.diag_indices_from(G)] -= 1.0
    return float(np.linalg.norm(G))


def residual(A: np.ndarray, Q: np.ndarray, R: np.ndarray, block: int = 1 << 18) -> float:
    """||Q R - A||_F / ||A||_F, accumulated over row blocks."""
    num = 0.0
    den = 0.0
    for r0 in range(0, A.shape[0], block):
        a = A[r0:r0 + block]
        d = Q[r0:r0 + block] @ R - a
        num += float(np.sum(d * d))
        den += float(np.sum(a * a))
    return math.sqrt(num) / math.sqrt(den)


def rel_error(X: np.ndarray, X_ref: np.ndarray) -> float:
    """||X - X_ref||_F / ||X_ref||_F."""
    return float(np.linalg.norm(X - X_ref) / np.linalg.norm(X_ref))


def nominal_flops(m: int, n: int) -> float:
    """Flops of CQR2 as the paper counts them (Section IV): 4 m n^2 + 5 n^3 / 3."""
    return 4.0 * m * n * n + 5.0 * n ** 3 / 3.0
