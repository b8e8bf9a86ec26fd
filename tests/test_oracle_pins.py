"""Pins of the CPU FP64 oracle against facts that do not come from the oracle.

* exact closed forms for CholInv (min(i,j) and Pascal matrices, golden files);
* brute force: an independent Householder QR, itself checked against LAPACK;
* closed forms for CQR2: A = U R0, n = 1, orthonormal A, A = U diag(d);
* invariants: Q^T Q = I, Q R = A, R upper with positive diagonal, and the
  kappa^2 law of the first CholeskyQR pass against the O(eps) second pass
  (Section I);
* least squares against a consistent system and the normal equations;
* breakdown reporting;
* planted mistakes: mutated copies of the oracle must fail these pins.
"""
from __future__ import annotations

import inspect
import math
import types

import numpy as np
import pytest

import oracle
import oracle.cholqr2 as ocq
import synth
from closed_forms import minij, pascal, read_golden, upper_with_kappa

EPS = 2.0 ** -53


# ------------------------------------------------------------ CholInv pins

@pytest.mark.parametrize("name,gen", [("minij_n6.txt", minij), ("pascal_n5.txt", pascal)])
def test_cholinv_golden_fixture(name, gen):
    g = read_golden(name)
    n = g["W"].shape[0]
    W, L, Y = gen(n)
    np.testing.assert_array_equal(W, g["W"])
    np.testing.assert_array_equal(L, g["L"])
    np.testing.assert_array_equal(Y, g["Y"])
    Lo, Yo = oracle.cholinv(g["W"])
    np.testing.assert_array_equal(Lo, g["L"])
    np.testing.assert_array_equal(Yo, g["Y"])


@pytest.mark.parametrize("n", [1, 2, 3, 5, 7, 8, 13, 64, 100, 129, 257, 512])
def test_cholinv_minij_exact(n):
    W, L, Y = minij(n)
    Lo, Yo = oracle.cholinv(W)
    np.testing.assert_array_equal(Lo, L)
    np.testing.assert_array_equal(Yo, Y)


@pytest.mark.parametrize("n", [2, 3, 6, 9, 16, 21, 28])
def test_cholinv_pascal_exact(n):
    W, L, Y = pascal(n)
    Lo, Yo = oracle.cholinv(W)
    np.testing.assert_array_equal(Lo, L)
    np.testing.assert_array_equal(Yo, Y)


def test_cholinv_diagonal():
    d = np.array([4.0, 9.0, 0.25, 16.0, 1.0])
    Lo, Yo = oracle.cholinv(np.diag(d))
    np.testing.assert_array_equal(Lo, np.diag(np.sqrt(d)))
    np.testing.assert_array_equal(Yo, np.diag(1.0 / np.sqrt(d)))


@pytest.mark.parametrize("n", [1, 4, 31, 64, 97])
def test_cholinv_invariants_random_spd(n):
    A = synth.make_matrix(4 * n + 8, n, 1e3, seed=5)
    W = A.T @ A
    L, Y = oracle.cholinv(W)
    assert np.array_equal(L, np.tril(L)) and np.array_equal(Y, np.tril(Y))
    assert np.all(np.diag(L) > 0)
    assert np.linalg.norm(L @ L.T - W) <= 50 * n * EPS * np.linalg.norm(W)
    # Y = L^-1: both residuals, bounded by cond(L) * n * eps
    kl = np.linalg.cond(L)
    assert np.linalg.norm(L @ Y - np.eye(n)) <= 50 * n * kl * EPS
    assert np.linalg.norm(Y @ L - np.eye(n)) <= 50 * n * kl * EPS
    # agrees with LAPACK's Cholesky
    Lref = np.linalg.cholesky(W)
    assert np.linalg.norm(L - Lref) <= 50 * n * kl * EPS * np.linalg.norm(Lref)


def test_cholinv_breakdown_index():
    W = np.diag([1.0, 2.0, -1.0, 3.0])
    with pytest.raises(oracle.NotSPD) as e:
        oracle.cholinv(W)
    assert e.value.pivot == 2
    W = np.diag([1.0, 2.0, 3.0, 0.0, 5.0])
    with pytest.raises(oracle.NotSPD) as e:
        oracle.cholinv(W)
    assert e.value.pivot == 3
    W = np.eye(3)
    W[1, 1] = np.nan
    with pytest.raises(oracle.NotSPD) as e:
        oracle.cholinv(W)
    assert e.value.pivot == 1


# ------------------------------------------------ Householder (brute force)

@pytest.mark.parametrize("m,n", [(5, 1), (8, 8), (40, 7), (256, 32)])
def test_householder_matches_lapack(m, n):
    A = synth.make_matrix(m, n, None, seed=11)
    Q, R = oracle.householder_qr(A)
    Ql, Rl = np.linalg.qr(A)
    d = np.sign(np.diag(Rl))
    Ql, Rl = Ql * d, d[:, None] * Rl
    assert np.linalg.norm(R - Rl) <= 1e-13 * np.linalg.norm(Rl)
    assert np.linalg.norm(Q - Ql) <= 1e-13 * math.sqrt(n)
    assert np.all(np.diag(R) > 0)


@pytest.mark.parametrize("m,n,kappa", [(16, 4, None), (64, 16, 1e2), (256, 32, 1e4), (200, 31, 1e3),
                                       (32, 32, 10.0)])
def test_cqr2_matches_householder(m, n, kappa):
    A = synth.make_matrix(m, n, kappa, seed=3)
    Q, R = oracle.cqr2(A)
    Qh, Rh = oracle.householder_qr(A)
    k = kappa or 10.0
    tol = 10 * n * k * EPS
    assert oracle.rel_error(R, Rh) <= tol
    assert np.linalg.norm(Q - Qh) / math.sqrt(n) <= tol


# ------------------------------------------------------- CQR2 closed forms

def test_cqr2_n1():
    a = synth.make_matrix(1000, 1, None, seed=2)
    Q, R = oracle.cqr2(a)
    nrm = np.linalg.norm(a[:, 0])
    assert abs(R[0, 0] - nrm) <= 4 * EPS * nrm
    assert np.max(np.abs(Q[:, 0] - a[:, 0] / nrm)) <= 8 * EPS


@pytest.mark.parametrize("m,n,kappa", [(300, 20, 10.0), (1000, 50, 1e4), (4096, 64, 1e6)])
def test_cqr2_recovers_U_R0(m, n, kappa):
    U = synth.random_orthogonal(m, seed=9)[:, :n]
    R0 = upper_with_kappa(n, kappa, seed=4)
    A = U @ R0
    Q, R = oracle.cqr2(A)
    kr = np.linalg.cond(R0)
    assert oracle.rel_error(R, R0) <= 20 * n * kr * EPS
    assert np.linalg.norm(Q - U) <= 20 * n * kr * EPS


def test_cqr2_orthonormal_input_gives_identity():
    U = synth.random_orthogonal(512, seed=8)[:, :40]
    Q, R = oracle.cqr2(U)
    assert np.linalg.norm(R - np.eye(40)) <= 100 * EPS * 40
    assert np.linalg.norm(Q - U) <= 100 * EPS * 40


def test_cqr2_scaled_orthonormal_gives_diag():
    U = synth.random_orthogonal(256, seed=12)[:, :16]
    d = np.logspace(2, -2, 16)
    Q, R = oracle.cqr2(U * d)
    assert np.linalg.norm(R - np.diag(d)) <= 100 * 16 * 1e4 * EPS * np.linalg.norm(d)
    assert np.linalg.norm(Q - U) <= 100 * 16 * 1e4 * EPS


# ------------------------------------------------------------- invariants

@pytest.mark.parametrize("kappa", [None, 1e2, 1e4, 1e6])
def test_cqr2_invariants(kappa):
    m, n = 4096, 64
    A = synth.make_matrix(m, n, kappa, seed=1)
    Q, R, info = oracle.cqr2(A, keep=True)
    assert np.array_equal(R, np.triu(R))
    assert np.all(np.diag(R) > 0)
    assert oracle.orthogonality(Q) <= 1e-13
    assert oracle.residual(A, Q, R) <= 1e-14
    # Section I: CholeskyQR's Q has error Theta(kappa^2 eps); the second pass
    # factors a nearly orthogonal Q1 so R2 is near identity.
    k = kappa or 1.3
    o1 = oracle.orthogonality(info["Q1"])
    assert o1 <= 10 * n * k * k * EPS
    assert np.linalg.norm(info["R2"] - np.eye(n)) <= 10 * n * k * k * EPS


def test_first_pass_error_grows_as_kappa_squared():
    m, n = 4096, 32
    o1 = []
    for kappa in (1e3, 1e5):
        A = synth.make_matrix(m, n, kappa, seed=21)
        _, _, info = oracle.cqr2(A, keep=True)
        o1.append(oracle.orthogonality(info["Q1"]))
    ratio = o1[1] / o1[0]
    # kappa grows 100x, so the first-pass loss of orthogonality grows ~1e4x
    assert 1e3 <= ratio <= 1e5, ratio


def test_cqr2_breakdown_reports_pass():
    A = synth.make_matrix(100, 6, None, seed=3)
    A[:, 4] = 0.0
    with pytest.raises(oracle.PassFailed) as e:
        oracle.cqr2(A)
    assert e.value.pass_no == 1 and e.value.pivot == 4


def test_cqr2_rejects_wide():
    with pytest.raises(ValueError):
        oracle.cqr2(np.ones((3, 5)))


# --------------------------------------------------------- least squares

def test_lstsq_consistent_system():
    A = synth.make_matrix(2000, 48, 1e4, seed=31)
    x0 = np.linspace(-1, 1, 48)
    b = A @ x0
    x = oracle.lstsq(A, b)
    assert np.linalg.norm(x - x0) <= 100 * 48 * 1e4 * EPS * np.linalg.norm(x0)


def test_lstsq_normal_equations():
    A = synth.make_matrix(3000, 40, 1e3, seed=32)
    b = synth.make_rhs(3000, seed=32)
    x = oracle.lstsq(A, b)
    r = A @ x - b
    assert np.linalg.norm(A.T @ r) <= 1e-12 * np.linalg.norm(A) * np.linalg.norm(r)
    xl = np.linalg.lstsq(A, b, rcond=None)[0]
    assert np.linalg.norm(x - xl) <= 1e-10 * np.linalg.norm(xl)


def test_back_substitution_exact():
    R = np.array([[2.0, 1.0, -1.0], [0.0, 4.0, 2.0], [0.0, 0.0, 0.5]])
    x = np.array([1.0, -2.0, 4.0])
    np.testing.assert_array_equal(oracle.back_substitution(R, R @ x), x)


def test_nominal_flops():
    # Section IV: 4 m n^2 + 5 n^3 / 3
    assert oracle.nominal_flops(4096, 64) == 4 * 4096 * 64 * 64 + 5 * 64 ** 3 / 3


# ------------------------------------------------------ planted mistakes

_MUTATIONS = {
    "y21_sign": ("Y21 = -(Y22 @ U)", "Y21 = (Y22 @ U)"),
    "l21_no_transpose": ("L21 = A21 @ Y11.T", "L21 = A21 @ Y11"),
    "schur_dropped": ("_cholinv(A22 - L21 @ L21.T, offset + n1)", "_cholinv(A22, offset + n1)"),
    "u_wrong_order": ("U = L21 @ Y11", "U = Y11.T @ L21.T @ Y11.T @ Y11"),
    "split_index": ("A21 = A[n1:, :n1]", "A21 = A[n1:, :n1].copy(); A21[:, 0] = A[n1:, 1]"),
    "base_inverse": ("np.array([[1.0 / l]])", "np.array([[1.0 / a]])"),
    "qform_transposed": ("Q = A @ Rinv", "Q = A @ Rinv.T"),
    "r_order": ("R = np.triu(R2 @ R1)", "R = np.triu(R1 @ R2)"),
}


def _mutant(key: str) -> types.ModuleType:
    src = inspect.getsource(ocq)
    old, new = _MUTATIONS[key]
    assert src.count(old) == 1, key
    mod = types.ModuleType(f"oracle_mutant_{key}")
    exec(compile(src.replace(old, new), f"<mutant {key}>", "exec"), mod.__dict__)
    return mod


def _pins_pass(mod) -> bool:
    """The core pins, run against a (possibly mutated) oracle module."""
    try:
        for n in (6, 9):
            W, L, Y = pascal(n)
            Lo, Yo = mod.cholinv(W)
            if not (np.array_equal(Lo, L) and np.array_equal(Yo, Y)):
                return False
        ok = True
        # kappa 1e6 makes R2 visibly different from I, so R1 R2 != R2 R1
        for kappa, tol in ((1e2, 1e-12), (1e6, 1e-8)):
            A = synth.make_matrix(64, 8, kappa, seed=3)
            Q, R = mod.cqr2(A)
            Qh, Rh = oracle.householder_qr(A)
            ok = ok and bool(np.linalg.norm(R - Rh) <= tol * np.linalg.norm(Rh)
                             and np.linalg.norm(Q - Qh) <= tol)
        return ok
    except Exception:
        return False


def test_pins_accept_oracle():
    assert _pins_pass(ocq)


@pytest.mark.parametrize("key", sorted(_MUTATIONS))
def test_pins_reject_planted_mistake(key):
    assert not _pins_pass(_mutant(key))


# ------------------------------------------- shifted CholeskyQR3 (NEXT row)

def test_shift_formula():
    A = synth.make_matrix(300, 12, 1e3, seed=41)
    W = oracle.syrk(A)
    s = oracle.shift_of(W, 300)
    assert s == pytest.approx(11 * (300 * 12 + 12 * 13) * EPS * np.linalg.norm(A) ** 2, rel=1e-12)


@pytest.mark.parametrize("kappa", [1e2, 1e6, 1e9, 1e12])
def test_scqr3_unconditionally_stable(kappa):
    m, n = 4096, 48
    A = synth.make_matrix(m, n, kappa, seed=42)
    Q, R = oracle.scqr3(A)
    assert np.array_equal(R, np.triu(R)) and np.all(np.diag(R) > 0)
    assert oracle.orthogonality(Q) <= 100 * n * EPS
    assert oracle.residual(A, Q, R) <= 100 * n * EPS
    Qh, Rh = oracle.householder_qr(A)
    # both are backward stable: R agrees with Householder's far better than kappa eps
    assert oracle.rel_error(R, Rh) <= 1e-12


def test_scqr3_where_cqr2_breaks_down():
    A = synth.make_matrix(2048, 32, 1e10, seed=43)
    with pytest.raises(oracle.NotSPD):
        oracle.cqr2(A)
    Q, R = oracle.scqr3(A)
    assert oracle.orthogonality(Q) <= 100 * 32 * EPS


def test_scqr3_needs_the_shift():
    # planted mistake: without the shift the first pass breaks down at kappa 1e10
    A = synth.make_matrix(2048, 32, 1e10, seed=43)
    src = inspect.getsource(ocq)
    old = "    Ws = W + s * np.eye(W.shape[0])"
    assert src.count(old) == 1
    mod = types.ModuleType("oracle_mutant_noshift")
    exec(compile(src.replace(old, "    Ws = W"), "<mutant noshift>", "exec"), mod.__dict__)
    with pytest.raises(mod.NotSPD):
        mod.scqr3(A)


# ------------------------------- inverse depth (Section III-A, InverseDepth)

def _leaf_mask(n: int, depth: int) -> np.ndarray:
    """True on the diagonal blocks of a depth-`depth` halving (split n // 2)."""
    M = np.zeros((n, n), dtype=bool)

    def rec(o, k, d):
        if d == 0 or k == 1:
            M[o:o + k, o:o + k] = True
            return
        k1 = k // 2
        rec(o, k1, d - 1)
        rec(o + k1, k - k1, d - 1)

    rec(0, n, depth)
    return M


@pytest.mark.parametrize("n,depth", [(8, 1), (8, 3), (13, 2), (64, 4), (100, 3), (129, 5)])
def test_cholinv_depth_minij_exact(n, depth):
    # integer closed form: L = all-ones lower triangle exactly, and the inverse
    # kept only on the leaf diagonal blocks (exact bidiagonal blocks of L^-1)
    W, L, Y = minij(n)
    Lo, Yo = oracle.cholinv_depth(W, depth)
    np.testing.assert_array_equal(Lo, L)
    np.testing.assert_array_equal(Yo, np.where(_leaf_mask(n, depth), Y, 0.0))


@pytest.mark.parametrize("depth", [0, 1, 2, 3, 6])
def test_right_solve_defining_property(depth):
    # X = B L^-T means X L^T = B; L and its inverse come from LAPACK, not the oracle
    rng = np.random.default_rng(depth)
    n, M = 150, 40
    G = rng.standard_normal((n, n))
    L = np.linalg.cholesky(G @ G.T + n * np.eye(n))
    X = oracle.right_solve(rng.standard_normal((M, n)), L, np.linalg.inv(L), depth)
    B = X @ L.T
    assert np.linalg.norm(oracle.right_solve(B, L, np.linalg.inv(L), depth) - X) <= 1e-12 * np.linalg.norm(X)
    B2 = rng.standard_normal((M, n))
    X2 = oracle.right_solve(B2, L, np.linalg.inv(L), depth)
    assert np.linalg.norm(X2 @ L.T - B2) <= 1e-13 * np.linalg.norm(B2)


@pytest.mark.parametrize("m,n,kappa,depth", [(400, 64, 1e3, 1), (400, 64, 1e3, 3), (900, 150, 1e6, 2),
                                             (300, 33, 1e4, 5)])
def test_cqr2_depth_matches_householder(m, n, kappa, depth):
    A = synth.make_matrix(m, n, kappa, seed=5)
    Q, R = oracle.cqr2(A, inverse_depth=depth)
    Qh, Rh = oracle.householder_qr(A)
    tol = 10 * n * kappa * EPS
    assert oracle.rel_error(R, Rh) <= tol
    assert np.linalg.norm(Q - Qh) / math.sqrt(n) <= tol
    assert oracle.orthogonality(Q) <= 100 * n * EPS


def test_right_solve_planted_missing_update_is_caught():
    # dropping the X1 L21^T term of the block substitution (a plausible slip)
    src = inspect.getsource(ocq)
    old = "    X2 = right_solve(B[:, n1:] - X1 @ L[n1:, :n1].T, L[n1:, n1:], Y[n1:, n1:], depth - 1)"
    assert src.count(old) == 1
    mod = types.ModuleType("oracle_mutant_noupdate")
    exec(compile(src.replace(old, old.replace(" - X1 @ L[n1:, :n1].T", "")), "<mutant noupdate>", "exec"),
         mod.__dict__)
    W, L, Y = minij(20)
    try:
        Lm, _ = mod.cholinv_depth(W, 2)
        assert not np.array_equal(Lm, L)
    except mod.NotSPD:
        pass  # the wrong Schur complement broke down: caught as well
    B = np.random.default_rng(1).standard_normal((30, 20))
    X = mod.right_solve(B, L, Y, 2)
    assert np.linalg.norm(X @ L.T - B) > 1e-3 * np.linalg.norm(B)


# ------------------------------------- the error norms every parity test uses
#
# orthogonality, residual and rel_error are the yardsticks of the GPU parity
# tests and of the bench's error report, so they are pinned to values fixed by
# exact arithmetic: dyadic inputs whose products and sums are exact in FP64,
# with the expected norms worked out in rational arithmetic (fractions), not by
# the functions under test.

from fractions import Fraction  # noqa: E402


def _hadamard(k: int) -> np.ndarray:
    """Sylvester Hadamard matrix of order 2^k (entries +-1, H^T H = 2^k I)."""
    H = np.ones((1, 1))
    for _ in range(k):
        H = np.block([[H, H], [H, -H]])
    return H


def _frob_exact(E) -> Fraction:
    """Squared Frobenius norm of a matrix of Fractions."""
    return sum((x * x for row in E for x in row), Fraction(0))


def _ortho_case():
    """Q = U M with U = H_16 / 4 (exactly orthonormal columns) and a dyadic
    upper-triangular M: Q^T Q - I = M^T M - I exactly."""
    U = _hadamard(4)[:, [1, 6, 11]] / 4.0
    Mf = [[Fraction(1), Fraction(1, 4), Fraction(0)],
          [Fraction(0), Fraction(1), Fraction(1, 2)],
          [Fraction(0), Fraction(0), Fraction(3, 4)]]
    M = np.array([[float(x) for x in r] for r in Mf])
    n = 3
    E = [[sum((Mf[k][i] * Mf[k][j] for k in range(n)), Fraction(0)) - (1 if i == j else 0) for j in range(n)]
         for i in range(n)]
    return U @ M, _frob_exact(E)


def test_orthogonality_exact_value():
    Q, e2 = _ortho_case()
    assert e2 == Fraction(170, 256)  # worked by hand: diag (0, 1/16, -3/16), off-diagonal 1/4, 1/2
    assert oracle.orthogonality(Q) == pytest.approx(math.sqrt(170) / 16, rel=4 * EPS)


def test_orthogonality_of_exactly_orthonormal_columns_is_zero():
    # columns with disjoint supports far apart (+-1/2 on four rows each)
    m = 3 * (1 << 18) + 5
    Q = np.zeros((m, 4))
    rows = [[0, 1 << 18, (1 << 19) + 3, m - 1], [5, 77, 1 << 17, m - 2], [9, 10, 11, 12], [m - 3, m - 4, 200, 300]]
    for j, rs in enumerate(rows):
        Q[rs, j] = [0.5, -0.5, 0.5, 0.5]
    assert oracle.orthogonality(Q) == 0.0
    Q[(1 << 19) + 3, 0] *= 2.0  # one entry doubled: column norm^2 1 + 3/4, nothing else changes
    assert oracle.orthogonality(Q) == pytest.approx(0.75, rel=2 * EPS)


def _residual_case(block_offsets):
    """A = Q R + E over several 2^18-row blocks and a ragged tail, with Q, R,
    E dyadic so that Q R is exact; returns (A, Q, R, exact residual^2)."""
    m, n = 3 * (1 << 18) + 5, 2
    i = np.arange(m)
    Q4 = np.stack([(i % 3) - 1, (i % 5) - 2], axis=1)  # 4 Q as integers
    Q = Q4 / 4.0
    R = np.array([[2.0, 1.0], [0.0, 4.0]])
    QR4 = Q4 @ R.astype(np.int64)  # 4 Q R, exact integers
    E4 = np.zeros((m, n), dtype=np.int64)  # 4 E
    for (r, c, v) in block_offsets:
        E4[r, c] = v
    A4 = QR4 + E4
    A = A4 / 4.0
    num = int(np.sum(E4 * E4))
    den = int(np.sum(A4 * A4))  # int64: no rounding
    return A, Q, R, Fraction(num, den)


# one entry of E in each 2^18-row block, past the middle of the block, and one
# in the ragged last rows
_E_ENTRIES = [(200_000, 0, 12), ((1 << 18) + 150_001, 1, -16), ((1 << 19) + 140_000, 0, 48),
              (3 * (1 << 18) + 4, 1, 4)]


def test_residual_exact_value_across_blocks():
    A, Q, R, r2 = _residual_case(_E_ENTRIES)
    want = math.sqrt(r2.numerator) / math.sqrt(r2.denominator)
    assert oracle.residual(A, Q, R) == pytest.approx(want, rel=8 * EPS)
    # the blocking is an implementation detail: any block size gives the same value
    assert oracle.residual(A, Q, R, block=1000) == pytest.approx(want, rel=8 * EPS)
    # and Q R = A gives exactly zero
    assert oracle.residual(Q @ R, Q, R) == 0.0


def test_rel_error_exact_values():
    X = synth.make_matrix(50, 7, 1e2, seed=61)
    assert oracle.rel_error(2.0 * X, X) == pytest.approx(1.0, rel=2 * EPS)
    assert oracle.rel_error(X, X) == 0.0
    # ||D||_F / ||Xr||_F with D and Xr dyadic: sqrt(9 + 16) / sqrt(4 + 1 + 4 + 16)
    Xr = np.array([[2.0, 0.0], [1.0, -2.0], [0.0, 4.0]])
    D = np.array([[0.0, 3.0], [0.0, 0.0], [-4.0, 0.0]])
    assert oracle.rel_error(Xr + D, Xr) == pytest.approx(1.0, rel=2 * EPS)
    assert oracle.rel_error(Xr + D / 5.0, Xr) == pytest.approx(0.2, rel=4 * EPS)


_YARDSTICK_MUTATIONS = {
    "ortho_no_identity": ("    G[np.diag_indices_from(G)] -= 1.0\n", ""),
    "ortho_outer_product": ("    G = Q.T @ Q\n", "    G = Q @ Q.T\n"),
    "ortho_two_norm": ("    return float(np.linalg.norm(G))", "    return float(np.linalg.norm(G, 2))"),
    "residual_unsquared": ("        num += float(np.sum(d * d))", "        num += float(np.sum(np.abs(d)))"),
    "residual_no_root_denominator": ("    return math.sqrt(num) / math.sqrt(den)", "    return math.sqrt(num) / den"),
    "residual_last_block_dropped": ("    for r0 in range(0, A.shape[0], block):",
                                    "    for r0 in range(0, A.shape[0] - block, block):"),
    "residual_half_blocks": ("        a = A[r0:r0 + block]\n        d = Q[r0:r0 + block] @ R - a",
                             "        a = A[r0:r0 + block // 2]\n        d = Q[r0:r0 + block // 2] @ R - a"),
    "rel_error_wrong_normaliser": ("np.linalg.norm(X - X_ref) / np.linalg.norm(X_ref)",
                                   "np.linalg.norm(X - X_ref) / np.linalg.norm(X)"),
}


def _yardstick_mutant(key: str) -> types.ModuleType:
    src = inspect.getsource(ocq)
    old, new = _YARDSTICK_MUTATIONS[key]
    assert src.count(old) == 1, key
    mod = types.ModuleType(f"oracle_mutant_{key}")
    exec(compile(src.replace(old, new), f"<mutant {key}>", "exec"), mod.__dict__)
    return mod


def _yardstick_pins_pass(mod) -> bool:
    try:
        Q, e2 = _ortho_case()
        if mod.orthogonality(Q) != pytest.approx(math.sqrt(170) / 16, rel=4 * EPS):
            return False
        A, Qr, R, r2 = _residual_case(_E_ENTRIES)
        if mod.residual(A, Qr, R) != pytest.approx(math.sqrt(r2.numerator) / math.sqrt(r2.denominator),
                                                     rel=8 * EPS):
            return False
        X = synth.make_matrix(50, 7, 1e2, seed=61)
        return mod.rel_error(2.0 * X, X) == pytest.approx(1.0, rel=2 * EPS)
    except Exception:
        return False


def test_yardstick_pins_accept_oracle():
    assert _yardstick_pins_pass(ocq)


@pytest.mark.parametrize("key", sorted(_YARDSTICK_MUTATIONS))
def test_yardstick_pins_reject_planted_mistake(key):
    assert not _yardstick_pins_pass(_yardstick_mutant(key))


# ------------------------------- CholeskyQR2 on column panels (Section V)

@pytest.mark.parametrize("m,n,b,kappa", [(600, 96, 32, 1e3), (1500, 300, 128, 1e5), (2048, 512, 128, 1e6),
                                         (400, 50, 1, 1e2), (777, 130, 64, 1e4)])
def test_panel_cqr2_matches_householder(m, n, b, kappa):
    A = synth.make_matrix(m, n, kappa, seed=51)
    Q, R = oracle.panel_cqr2(A, b)
    Qh, Rh = oracle.householder_qr(A)
    tol = 10 * n * kappa * EPS
    assert np.array_equal(R, np.triu(R)) and np.all(np.diag(R) > 0)
    assert oracle.rel_error(R, Rh) <= tol
    assert np.linalg.norm(Q - Qh) / math.sqrt(n) <= tol
    # the reorthogonalised projections keep Q orthonormal to working accuracy
    assert oracle.orthogonality(Q) <= 100 * n * EPS
    assert oracle.residual(A, Q, R) <= 100 * n * EPS


def test_panel_cqr2_one_panel_is_cqr2():
    A = synth.make_matrix(500, 40, 1e4, seed=52)
    for b in (40, 64, 1000):
        Q, R = oracle.panel_cqr2(A, b)
        Qc, Rc = oracle.cqr2(A)
        np.testing.assert_array_equal(Q, Qc)
        np.testing.assert_array_equal(R, Rc)


def test_panel_cqr2_breakdown_reports_column_of_A():
    A = synth.make_matrix(1000, 200, 1e2, seed=53)
    A[:, 150] = 0.0  # panel 2 of width 64 (columns 128..191)
    with pytest.raises(oracle.PassFailed) as e:
        oracle.panel_cqr2(A, 64)
    assert e.value.pass_no == 1 and e.value.pivot == 150


_PANEL_MUTATIONS = {
    "panel_no_reorthogonalisation": ("            for _ in range(2):  # projection, then reorthogonalisation",
                                     "            for _ in range(1):  # projection, then reorthogonalisation"),
    "panel_coefficients_overwritten": ("                R[:c0, c0:c1] += C", "                R[:c0, c0:c1] = C"),
    "panel_pivot_not_shifted": ("NotSPD(e.pivot + c0, e.value)", "NotSPD(e.pivot, e.value)"),
}


def _panel_pins_pass(mod) -> bool:
    try:
        A = synth.make_matrix(2048, 512, 1e6, seed=54)
        Q, R = mod.panel_cqr2(A, 128)
        Qh, Rh = oracle.householder_qr(A)
        if not (oracle.orthogonality(Q) <= 100 * 512 * EPS and oracle.residual(A, Q, R) <= 100 * 512 * EPS
                and oracle.rel_error(R, Rh) <= 10 * 512 * 1e6 * EPS):
            return False
        B = synth.make_matrix(1000, 200, 1e2, seed=53)
        B[:, 150] = 0.0
        try:
            mod.panel_cqr2(B, 64)
            return False
        except mod.PassFailed as e:
            return e.pivot == 150
    except Exception:
        return False


def test_panel_pins_accept_oracle():
    assert _panel_pins_pass(ocq)


@pytest.mark.parametrize("key", sorted(_PANEL_MUTATIONS))
def test_panel_pins_reject_planted_mistake(key):
    src = inspect.getsource(ocq)
    old, new = _PANEL_MUTATIONS[key]
    assert src.count(old) == 1, key
    mod = types.ModuleType(f"oracle_mutant_{key}")
    exec(compile(src.replace(old, new), f"<mutant {key}>", "exec"), mod.__dict__)
    assert not _panel_pins_pass(mod)
