"""Pins of the FP64 oracle against facts that do not come from the oracle itself:
published test vectors of the counter hash, exact rational arithmetic on small
inputs (the inputs are dyadic rationals, so the exact result is computable),
closed forms (identity and rank-1 products, known norms), invariants, and the
standard rounding-error bound of a dot product (|error| <= gamma_K |A||B|).
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
U = 2.0 ** -53  # unit roundoff of binary64


def _frac_matrix(X):
    return [[Fraction(float(v)) for v in row] for row in np.asarray(X, dtype=np.float64)]


def _frac_gemm(A, B, C0, alpha, beta):
    M, K, N = len(A), len(A[0]), len(B[0])
    a, b = Fraction(alpha), Fraction(beta)
    return [[a * sum(A[i][k] * B[k][j] for k in range(K)) + b * C0[i][j] for j in range(N)] for i in range(M)]


# ---- counter hash -------------------------------------------------------------

def test_splitmix64_published_vectors():
    want = [int(l, 16) for l in open(os.path.join(GOLDEN, "splitmix64_seed0.txt")) if l.startswith("0x")]
    got = [int(x) for x in oracle.splitmix64_stream(0, len(want))]
    assert got == want
    # first output of a generator in state s equals the one-shot hash of s
    assert oracle.splitmix64(0) == want[0]


def test_init_values_are_dyadic_in_range():
    X = oracle.init_matrix(1000, 0, 64, 96)
    assert X.min() >= -1.0 and X.max() < 1.0
    k = (X + 1.0) * 2.0 ** 23
    assert np.all(k == np.round(k)) and k.min() >= 0 and k.max() < 2 ** 24
    assert np.all(X.astype(np.float32).astype(np.float64) == X)  # exact in binary32


def test_init_moments_uniform():
    X = oracle.init_matrix(1001, 1, 1024, 1024).ravel()
    n = X.size
    # U[-1,1): mean 0 (sd 1/sqrt(3n)), variance 1/3 (sd of sample var ~ sqrt(4/45/n))
    assert abs(X.mean()) < 5 / math.sqrt(3 * n)
    assert abs(X.var() - 1 / 3) < 5 * math.sqrt(4 / 45 / n)
    # buffers and seeds give independent streams
    Y = oracle.init_matrix(1001, 2, 1024, 1024).ravel()
    assert abs(np.corrcoef(X, Y)[0, 1]) < 5 / math.sqrt(n)
    Z = oracle.init_matrix(1002, 1, 1024, 1024).ravel()
    assert abs(np.corrcoef(X, Z)[0, 1]) < 5 / math.sqrt(n)


def test_row_exponents_spread_and_exact_scaling():
    e = np.array([oracle.row_exponent(1003, i) for i in range(4096)])
    assert e.min() >= -10 and e.max() <= 10
    assert abs(e.mean()) < 0.5
    assert 2.5 < e.std() < 4.0  # Irwin-Hall(12) * 10/3, rounded
    assert e.min() <= -8 and e.max() >= 8  # spans about 1e-3 .. 1e3
    X = oracle.init_matrix(1003, 0, 16, 8, rowscale=True)
    Y = oracle.init_matrix(1003, 0, 16, 8, rowscale=False)
    for i in range(16):
        assert np.all(X[i] == Y[i] * 2.0 ** oracle.row_exponent(1003, i))


# ---- GEMM ---------------------------------------------------------------------

def test_gemm_identity():
    A = oracle.init_matrix(1, 0, 24, 24)
    C0 = oracle.init_matrix(1, 2, 24, 24)
    C = oracle.gemm(A, np.eye(24), C0, 1.5, 0.5)
    assert np.array_equal(C, 1.5 * A + 0.5 * C0)  # every term exact (dyadic, few bits)


def test_gemm_rank1_closed_form():
    rng = np.random.default_rng(5)
    M, K, N = 7, 5, 9
    u, v, w, z = (rng.integers(-8, 9, size=s).astype(np.float64) for s in (M, K, K, N))
    A, B = np.outer(u, v), np.outer(w, z)
    C0 = np.zeros((M, N))
    C = oracle.gemm(A, B, C0, 1.0, 0.0)
    assert np.array_equal(C, float(v @ w) * np.outer(u, z))  # (u v^T)(w z^T) = (v.w) u z^T


@pytest.mark.parametrize("shape", [(8, 8, 8), (3, 5, 7), (7, 1, 4), (1, 9, 2)])
def test_gemm_exact_rational_bruteforce(shape):
    M, K, N = shape
    A = oracle.init_matrix(7, 0, M, K)
    B = oracle.init_matrix(7, 1, K, N)
    C0 = oracle.init_matrix(7, 2, M, N)
    got = oracle.gemm(A, B, C0, 1.5, 0.5)
    exact = _frac_gemm(_frac_matrix(A), _frac_matrix(B), _frac_matrix(C0), 1.5, 0.5)
    # rounding bound of a length-K dot product plus the two scalings and the add
    gamma = (K + 3) * U / (1 - (K + 3) * U)
    scale = 1.5 * (np.abs(A) @ np.abs(B)) + 0.5 * np.abs(C0)
    for i in range(M):
        for j in range(N):
            assert abs(Fraction(float(got[i, j])) - exact[i][j]) <= Fraction(gamma * scale[i, j] + 1e-300)


def test_gemm_inplace_alias_and_beta_zero():
    A = oracle.init_matrix(3, 0, 6, 4)
    B = oracle.init_matrix(3, 1, 4, 5)
    C0 = oracle.init_matrix(3, 2, 6, 5)
    ref = oracle.gemm(A, B, np.zeros((6, 5)), 2.0, 0.0)
    exact = _frac_gemm(_frac_matrix(A), _frac_matrix(B), _frac_matrix(np.zeros((6, 5))), 2.0, 0.0)
    assert max(abs(float(Fraction(float(ref[i, j])) - exact[i][j])) for i in range(6) for j in range(5)) < 1e-14
    # beta C0 term enters with its sign and scale
    C = oracle.gemm(A, B, C0, 2.0, -0.25)
    assert np.allclose(C - ref, -0.25 * C0, rtol=0, atol=1e-14)


def test_gemm_sampled_entries_match_materialised():
    seed, M, N, K = 11, 40, 24, 33
    A = oracle.init_matrix(seed, 0, M, K, rowscale=True)
    B = oracle.init_matrix(seed, 1, K, N)
    C0 = oracle.init_matrix(seed, 2, M, N)
    full = oracle.gemm(A, B, C0, 1.5, 0.5)
    ii = np.array([0, 5, 39, 17, 22])
    jj = np.array([0, 23, 7, 11, 0])
    got = oracle.gemm_init_entries(seed, (0, 1, 2), True, M, N, K, 1.5, 0.5, ii, jj)
    assert np.allclose(got, full[ii, jj], rtol=1e-15, atol=0)
    col = oracle.gemm_column(A, B, C0, 1.5, 0.5, 7)
    assert np.allclose(col, full[:, 7], rtol=1e-15, atol=0)


def _freivalds(C, A, B, C0, alpha, beta, rng):
    """Relative residuals of Freivalds' identities C x = alpha A (B x) + beta C0 x and
    y^T C = alpha (y^T A) B + beta y^T C0 for random sign vectors x, y (Freivalds 1977): a
    wrong entry, a transposed operand or a dropped term leaves a residual of its own size,
    whatever the loop order that formed C."""
    x = rng.choice([-1.0, 1.0], size=C.shape[1])
    y = rng.choice([-1.0, 1.0], size=C.shape[0])
    right = alpha * (A @ (B @ x)) + beta * (C0 @ x)
    left = alpha * ((y @ A) @ B) + beta * (y @ C0)
    return (float(np.linalg.norm(C @ x - right) / np.linalg.norm(right)),
            float(np.linalg.norm(y @ C - left) / np.linalg.norm(left)))


def test_gemm_freivalds_rectangular():
    """The oracle GEMM on odd rectangular shapes with row-scaled A satisfies both Freivalds
    identities to binary64 rounding; planted mistakes in its output (one entry off by 1e-9 of
    the largest, the beta term dropped, the product transposed, the operands swapped) each
    break them."""
    rng = np.random.default_rng(5)
    seed, M, N, K = 21, 517, 263, 389
    A = oracle.init_matrix(seed, 0, M, K, rowscale=True)
    B = oracle.init_matrix(seed, 1, K, N)
    C0 = oracle.init_matrix(seed, 2, M, N)
    C = oracle.gemm(A, B, C0, 1.5, 0.5)
    assert max(_freivalds(C, A, B, C0, 1.5, 0.5, rng)) <= 1e-13
    bad = C.copy()
    bad[300, 17] += 1e-9 * np.abs(C).max()
    assert max(_freivalds(bad, A, B, C0, 1.5, 0.5, rng)) > 1e-12
    assert max(_freivalds(C - 0.5 * C0, A, B, C0, 1.5, 0.5, rng)) > 1e-10
    # square operands, where a transposed product has the right shape
    P, Q = oracle.init_matrix(seed, 3, 64, 64), oracle.init_matrix(seed, 4, 64, 64)
    Z = np.zeros((64, 64))
    Cpq = oracle.gemm(P, Q, Z, 1.0, 0.0)
    assert max(_freivalds(Cpq, P, Q, Z, 1.0, 0.0, rng)) <= 1e-13
    assert max(_freivalds(Cpq.T.copy(), P, Q, Z, 1.0, 0.0, rng)) > 1e-10
    assert max(_freivalds(oracle.gemm(Q, P, Z, 1.0, 0.0), P, Q, Z, 1.0, 0.0, rng)) > 1e-10


# ---- element-wise and reductions -----------------------------------------------

def test_axpy_exact():
    X = oracle.init_matrix(4, 0, 9, 11)
    Y = oracle.init_matrix(4, 1, 9, 11)
    for alpha in (2.0, -0.5, 0.25, 3.0):
        got = oracle.axpy(X, alpha, Y)
        for i in range(9):
            for j in range(11):
                ex = Fraction(float(X[i, j])) + Fraction(alpha) * Fraction(float(Y[i, j]))
                assert abs(Fraction(float(got[i, j])) - ex) <= abs(ex) * Fraction(U)


def test_transpose_involution_and_norm():
    X = oracle.init_matrix(5, 0, 13, 29)
    T = oracle.transpose(X)
    assert T.shape == (29, 13)
    assert np.array_equal(oracle.transpose(T), X)
    u = np.arange(1, 14, dtype=np.float64)
    v = np.arange(-3, 26, dtype=np.float64)
    assert np.array_equal(oracle.transpose(np.outer(u, v)), np.outer(v, u))
    assert oracle.frobenius(T) == oracle.frobenius(X)


def test_rowsum_total_and_rank1():
    X = oracle.init_matrix(6, 0, 17, 23)
    r = oracle.rowsum(X)
    assert r.shape == (17, 1)
    exact_total = sum(Fraction(float(v)) for v in X.ravel())
    assert abs(Fraction(float(r.sum())) - exact_total) < Fraction(1, 10 ** 12)
    u = np.arange(1, 18, dtype=np.float64)
    v = np.linspace(-1, 1, 23)
    v = np.round(v * 64) / 64
    assert np.allclose(oracle.rowsum(np.outer(u, v)).ravel(), u * v.sum(), rtol=1e-15, atol=1e-15)


def test_frobenius_closed_forms():
    for n in (1, 3, 64, 257):
        assert oracle.frobenius(np.eye(n)) == math.sqrt(n)
    u = np.array([3.0, 4.0, 12.0])  # norm 13
    z = np.array([1.0, 2.0, 2.0, 4.0])  # norm 5
    assert oracle.frobenius(np.outer(u, z)) == 65.0
    X = oracle.init_matrix(8, 0, 12, 10)
    exact = sum(Fraction(float(v)) ** 2 for v in X.ravel())
    got = Fraction(oracle.frobenius(X)) ** 2
    assert abs(got - exact) <= exact * Fraction(130 * U)


def test_relu_square_identities():
    X = oracle.init_matrix(9, 0, 10, 10)
    R = oracle.relu(X)
    assert np.all(R >= 0)
    assert np.array_equal(R - oracle.relu(-X), X)  # relu(x) - relu(-x) = x, exact
    S = oracle.square(X)
    for v, s in zip(X.ravel(), S.ravel()):
        ex = Fraction(float(v)) ** 2
        assert abs(Fraction(float(s)) - ex) <= ex * Fraction(U)
    u = np.array([1.0, -2.0, 0.5])
    v = np.array([3.0, -1.0])
    assert np.array_equal(oracle.square(np.outer(u, v)), np.outer(u * u, v * v))


def test_colmax_and_sum():
    X = oracle.init_matrix(10, 0, 31, 7)
    q = oracle.colmax(X)
    assert q.shape == (1, 7)
    assert np.array_equal(q.ravel(), X.max(axis=0))  # library routine
    perm = np.random.default_rng(1).permutation(31)
    assert np.array_equal(oracle.colmax(X[perm]), q)  # order-free
    u = np.array([1.0, 2.0, -4.0, 0.5])
    v = np.array([3.0, -1.0, 2.0])
    assert oracle.total(np.outer(u, v)) == float(u.sum() * v.sum())
    exact = sum(Fraction(float(v)) for v in X.ravel())
    assert abs(Fraction(oracle.total(X)) - exact) < Fraction(1, 10 ** 12)


# ---- whole programs ------------------------------------------------------------------

def test_six_loop_program_exact_n8():
    """End-to-end n=8 six-loop program against exact rational arithmetic."""
    prog = W.six_loop(8, seed=1000)
    out = oracle.run_program(prog)
    A = _frac_matrix(oracle.init_matrix(1000, 0, 8, 8))
    B = _frac_matrix(oracle.init_matrix(1000, 1, 8, 8))
    C0 = _frac_matrix(oracle.init_matrix(1000, 2, 8, 8))
    C = _frac_gemm(A, B, C0, 1.5, 0.5)
    D = [[C[i][j] + 2 * A[i][j] for j in range(8)] for i in range(8)]
    E = [[D[j][i] for j in range(8)] for i in range(8)]
    r = [sum(E[i]) for i in range(8)]
    f2 = sum(x * x for row in E for x in row)
    assert oracle.rel_err(out["C"], np.array([[float(x) for x in row] for row in C])) < 1e-15
    assert oracle.rel_err(out["E"], np.array([[float(x) for x in row] for row in E])) < 1e-15
    assert oracle.rel_err(out["r"].ravel(), np.array([float(x) for x in r])) < 1e-14
    assert abs(out["f"] ** 2 - float(f2)) / float(f2) < 1e-14


def test_twelve_loop_program_exact_small():
    prog = W.twelve_loop(6, 4, seed=1005)
    out = oracle.run_program(prog)
    A = oracle.init_matrix(1005, 0, 6, 4)
    B = oracle.init_matrix(1005, 1, 4, 6)
    C0 = oracle.init_matrix(1005, 2, 6, 6)
    S = oracle.init_matrix(1005, 3, 6, 6)
    Fa, Fb, Fc, Fs = map(_frac_matrix, (A, B, C0, S))
    C = _frac_gemm(Fa, Fb, Fc, 1.5, 0.5)
    D = [[C[i][j] + 2 * Fs[i][j] for j in range(6)] for i in range(6)]
    E = [[D[j][i] for j in range(6)] for i in range(6)]
    F = [[max(x, Fraction(0)) for x in row] for row in E]
    G = [[E[i][j] - Fraction(1, 2) * F[i][j] for j in range(6)] for i in range(6)]
    H = [[x * x for x in row] for row in G]
    P = [[H[i][j] + Fraction(1, 4) * D[i][j] for j in range(6)] for i in range(6)]
    q = [max(P[i][j] for i in range(6)) for j in range(6)]
    s = sum(x for row in P for x in row)
    fl = lambda M_: np.array([[float(x) for x in row] for row in M_])
    assert oracle.rel_err(out["P"], fl(P)) < 1e-14
    assert np.allclose(out["q"].ravel(), [float(x) for x in q], rtol=1e-14, atol=0)
    assert abs(out["s"] - float(s)) <= 1e-13 * float(sum(abs(x) for row in P for x in row))


def test_host_input_program_matches_six_loop():
    n, seed = 16, 77
    six = oracle.run_program(W.six_loop(n, seed))
    hp = W.host_input_program(n, seed)
    ins = {"A": oracle.init_matrix(seed, 0, n, n), "B": oracle.init_matrix(seed, 1, n, n),
           "C0": oracle.init_matrix(seed, 2, n, n)}
    out = oracle.run_program(hp, ins)
    assert np.array_equal(out["C"], six["C"]) and np.array_equal(out["r"], six["r"]) and out["f"] == six["f"]



def test_gemm_only_program_is_the_six_loop_gemm():
    """The GEMM-only workload computes the six-loop program's C (same buffers and hash
    streams), with and without row-scaled A."""
    for n, seed, rows in ((16, 77, False), (33, 78, True)):
        six = oracle.run_program(W.six_loop(n, seed, rowscale_a=rows, outputs=("C",)))
        out = oracle.run_program(W.gemm_only(n, seed, rowscale_a=rows))
        assert np.array_equal(out["C"], six["C"])

# ---- stencil loops (second workload) ------------------------------------------------------

def test_stencil_closed_forms():
    r, c = 11, 13
    const = np.full((r, c), 0.75)
    B = oracle.stencil3(const, 0)
    assert np.array_equal(B[1:-1, 1:-1], const[1:-1, 1:-1])  # weights sum to 1
    assert B[0, 0] == 0.75 * 9 / 16 and B[0, 5] == 0.75 * 12 / 16  # corner, edge with zero padding
    yy, xx = np.mgrid[0:r, 0:c].astype(np.float64)
    ramp = 3.0 * xx - 2.0 * yy + 1.0
    assert np.all(oracle.stencil3(ramp, 1)[1:-1, 1:-1] == 0.0)  # Laplacian of a linear function
    assert np.all(oracle.stencil3(ramp, 2)[1:-1, 1:-1] == 8.0 * 3.0)  # Sobel x: 2 * (1+2+1) * slope
    assert np.all(oracle.stencil3(ramp, 3)[1:-1, 1:-1] == 8.0 * -2.0)
    with pytest.raises(ValueError):
        oracle.stencil3(const, 7)


def test_stencil_exact_rational_and_adjoint():
    X = oracle.init_matrix(21, 0, 7, 9)
    Wt = [[Fraction(1, 16), Fraction(2, 16), Fraction(1, 16)], [Fraction(2, 16), Fraction(4, 16), Fraction(2, 16)],
         [Fraction(1, 16), Fraction(2, 16), Fraction(1, 16)]]
    F = _frac_matrix(X)
    got = oracle.stencil3(X, 0)
    for i in range(7):
        for j in range(9):
            ex = sum(Wt[a + 1][b + 1] * F[i + a][j + b] for a in (-1, 0, 1) for b in (-1, 0, 1)
                     if 0 <= i + a < 7 and 0 <= j + b < 9)
            assert abs(Fraction(float(got[i, j])) - ex) <= Fraction(10 * U) * 2
    # the symmetric presets are self-adjoint: <S x, y> = <x, S y>; Sobel-x is anti-symmetric
    Y = oracle.init_matrix(21, 1, 7, 9)
    for preset, sign in ((0, 1.0), (1, 1.0), (2, -1.0), (3, -1.0)):
        lhs = float((oracle.stencil3(X, preset) * Y).sum())
        rhs = sign * float((X * oracle.stencil3(Y, preset)).sum())
        assert abs(lhs - rhs) < 1e-12


def test_image_program_exact_small():
    prog = W.image_program(6, 7, seed=9, outputs=("B", "gx", "M2", "e", "q"))
    out = oracle.run_program(prog)
    X = oracle.init_matrix(9, 0, 6, 7)
    B = oracle.stencil3(X, 0)
    gx, gy = oracle.stencil3(B, 2), oracle.stencil3(B, 3)
    M2 = gx * gx + gy * gy
    assert np.array_equal(out["B"], B) and np.array_equal(out["gx"], gx)
    assert np.allclose(out["M2"], M2, rtol=1e-15, atol=0)
    assert abs(out["e"] - float(M2.sum())) <= 1e-13 * float(M2.sum())
    assert np.array_equal(out["q"].ravel(), out["M2"].max(axis=0))


# ---- loops Sec. 4 keeps on the CPU (dependence, early exit) -----------------------------

def test_recurrence_closed_forms():
    rng = np.random.default_rng(12)
    Xi = rng.integers(-50, 51, size=(6, 40)).astype(np.float64)
    assert np.array_equal(oracle.recurrence(Xi, 1.0), np.cumsum(Xi, axis=1))  # prefix sums, exact
    assert np.array_equal(oracle.recurrence(Xi, 0.0), Xi)
    E = np.zeros((2, 30))
    E[:, 0] = 1.0
    assert np.array_equal(oracle.recurrence(E, 0.5)[0], 0.5 ** np.arange(30))  # impulse response
    ones = np.ones((1, 40))
    assert np.array_equal(oracle.recurrence(ones, 2.0)[0], 2.0 ** (np.arange(40) + 1) - 1)  # geometric series
    assert oracle.recurrence(np.zeros((0, 5)), 1.0).shape == (0, 5)


def test_recurrence_exact_rational_bound():
    X = oracle.init_matrix(22, 0, 3, 25)
    alpha = 1.5
    got = oracle.recurrence(X, alpha)
    for i in range(3):
        y, scale = Fraction(0), 0.0
        for j in range(25):
            y = Fraction(float(X[i, j])) if j == 0 else Fraction(alpha) * y + Fraction(float(X[i, j]))
            scale = abs(float(X[i, j])) if j == 0 else alpha * scale + abs(float(X[i, j]))
            bound = 2 * (j + 1) * U / (1 - 2 * (j + 1) * U) * scale
            assert abs(Fraction(float(got[i, j])) - y) <= Fraction(bound)


def test_find_first_bruteforce_and_binary32_threshold():
    X = oracle.init_matrix(23, 0, 9, 17)
    for t in (-2.0, -0.5, 0.0, 0.7, 0.99, 1.0):
        got = oracle.find_first(X, t)
        for i in range(9):
            hits = [j for j in range(17) if X[i, j] > t]
            assert got[i, 0] == (hits[0] if hits else 17)
    # the threshold is the binary32 value of alpha: a binary32 0.1 does not exceed 0.1
    v = float(np.float32(0.1))
    row = np.array([[0.0, v, 1.0]])
    assert oracle.find_first(row, 0.1)[0, 0] == 2
    assert oracle.find_first(row, 0.0999)[0, 0] == 1
    assert oracle.find_first(np.zeros((2, 0)), 0.0)[0, 0] == 0  # empty rows: cols


def test_program_with_host_only_loops_exact_small():
    prog = W.analysis_program(6, 7, seed=5, outputs=("R", "C", "k", "s"))
    out = oracle.run_program(prog)
    X = oracle.init_matrix(5, 0, 6, 7)
    Bm = oracle.init_matrix(5, 1, 7, 7)
    R = oracle.recurrence(X, W.ANALYSIS_ALPHA)
    C = oracle.gemm(R, Bm, np.zeros((6, 7)), 1.0, 0.0)
    assert np.array_equal(out["R"], R) and np.array_equal(out["C"], C)
    k = oracle.find_first(C.T, W.ANALYSIS_THRESHOLD)
    assert np.array_equal(out["k"], k)
    assert out["s"] == oracle.total(np.maximum(C.T, 0.0))
