"""Pins of the FP64 oracle against what the paper and plain mathematics fix.

None of these compares the oracle with itself: every expected value comes
from a different route (brute-force sums, the Kronecker form, a library
routine, a closed form, or a value printed in the paper).
"""
import os

import numpy as np
import pytest
import scipy.linalg

import oracle
import workloads as W

RNG = np.random.default_rng(12345)


def rand(*shape):
    return np.asfortranarray(RNG.standard_normal(shape))


# ---------------------------------------------------------------- Tucker ---

@pytest.mark.parametrize("m,n", [
    ((1,), (3,)), ((3,), (1,)), ((2, 3), (4, 1)), ((3, 2, 4), (2, 4, 3)),
    ((1, 4, 1), (3, 1, 2)), ((2, 3, 2, 2), (3, 2, 1, 4)), ((4, 4, 4), (4, 4, 4)),
])
def test_tucker_equals_nested_sum(m, n):
    """Eq. (nestedmumode): brute-force sum over all input multi-indices."""
    T = rand(*m)
    Ls = [rand(n[k], m[k]) for k in range(len(m))]
    S = oracle.tucker(T, Ls)
    S2 = oracle.tucker_nested(T, Ls)
    assert S.shape == tuple(n)
    np.testing.assert_allclose(S, S2, rtol=1e-13, atol=1e-13 * np.abs(S2).max())


@pytest.mark.parametrize("m,n", [((3, 4, 5), (5, 2, 3)), ((4, 4, 4, 4), (4, 3, 2, 4)),
                                 ((7,), (5,)), ((6, 9), (8, 4))])
def test_tucker_equals_kronecker_form(m, n):
    """Lemma (krontomu): vec(S) = (L_d (x) ... (x) L_1) vec(T), the Kronecker
    product built with numpy.kron (a library routine, Appendix A definition)."""
    T = rand(*m)
    Ls = [rand(n[k], m[k]) for k in range(len(m))]
    K = Ls[0]
    for L in Ls[1:]:
        K = np.kron(L, K)
    ref = K @ oracle.vec(T)
    S = oracle.tucker(T, Ls)
    np.testing.assert_allclose(oracle.vec(S), ref, rtol=1e-12, atol=1e-12 * np.abs(ref).max())


def test_kron_matches_numpy():
    A, B = rand(3, 2), rand(4, 5)
    np.testing.assert_array_equal(oracle.kron(A, B), np.kron(A, B))


def test_identity_is_neutral():
    """The identity is the neutral element of the mu-mode product (Section 2)."""
    T = rand(5, 3, 4)
    S = oracle.tucker(T, [np.eye(5), np.eye(3), np.eye(4)])
    np.testing.assert_array_equal(S, T)


def test_products_in_distinct_modes_commute():
    """Order invariance of the Tucker operator (Section 2, after Eq. (nestedmumode))."""
    T = rand(4, 5, 6)
    A, B = rand(3, 4), rand(7, 6)
    S1 = oracle.mump(oracle.mump(T, A, 0), B, 2)
    S2 = oracle.mump(oracle.mump(T, B, 2), A, 0)
    np.testing.assert_allclose(S1, S2, rtol=1e-13, atol=1e-13)


def test_two_dimensional_case_is_matrix_product():
    """Eq. (gen2dmatmat): for d = 2, S = L_1 T L_2^T."""
    T = rand(6, 9)
    L1, L2 = rand(5, 6), rand(4, 9)
    np.testing.assert_allclose(oracle.tucker(T, [L1, L2]), L1 @ T @ L2.T, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("mu", [0, 1, 2, 3])
def test_mump_matches_tensordot(mu):
    """Definition (mmp): L applied to every mu-fibre, via numpy.tensordot."""
    T = rand(3, 4, 5, 2)
    L = rand(6, T.shape[mu])
    ref = np.moveaxis(np.tensordot(L, T, axes=([1], [mu])), 0, mu)
    np.testing.assert_allclose(oracle.mump(T, L, mu), ref, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(oracle.mump(T, np.asfortranarray(L.T), mu, transL=True), ref,
                               rtol=1e-13, atol=1e-13)


def test_rank_one_tensor():
    """T = a o b o c gives S = (L_1 a) o (L_2 b) o (L_3 c) (Eq. (nestedmumode) factorises)."""
    a, b, c = rand(7), rand(5), rand(6)
    T = np.asfortranarray(np.multiply.outer(np.multiply.outer(a, b), c))
    Ls = [rand(4, 7), rand(8, 5), rand(3, 6)]
    ref = np.multiply.outer(np.multiply.outer(Ls[0] @ a, Ls[1] @ b), Ls[2] @ c)
    np.testing.assert_allclose(oracle.tucker(T, Ls), ref, rtol=1e-13, atol=1e-13)


def test_kronsumv_matches_kronecker_sum():
    """Eq. (actkron) against the assembled Kronecker sum (Appendix A definition)."""
    n = (3, 4, 2)
    V = rand(*n)
    Ls = [rand(k, k) for k in n]
    K = np.zeros((int(np.prod(n)),) * 2)
    for mu in range(3):
        term = np.eye(1)
        for k in range(3):
            term = np.kron(Ls[k] if k == mu else np.eye(n[k]), term)
        K += term
    np.testing.assert_allclose(oracle.vec(oracle.kronsumv(V, Ls)), K @ oracle.vec(V),
                               rtol=1e-13, atol=1e-13)


# --------------------------------------------------------------- adjoint ---

def test_adjoint_dot_product():
    """<tucker(T), W> = <T, W x_mu L_mu^T> (Appendix A, property 5)."""
    m, n = (4, 5, 3), (6, 2, 4)
    T, Wt = rand(*m), rand(*n)
    Ls = [rand(n[k], m[k]) for k in range(3)]
    dT, _ = oracle.tucker_adjoint(T, Ls, Wt, want_dL=False)
    lhs = np.sum(oracle.tucker(T, Ls) * Wt)
    rhs = np.sum(T * dT)
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))


def _loss(T, Ls, target):
    r = oracle.tucker(T, Ls) - target
    return 0.5 * float(np.sum(r * r))


def test_adjoint_central_differences():
    """Gradient of 0.5 ||tucker(T, L) - target||^2 against central differences.
    The loss is quadratic along a single-argument direction, so central
    differences carry no truncation error."""
    m, n = (3, 4, 2, 3), (2, 3, 4, 3)
    T, target = rand(*m), rand(*n)
    Ls = [rand(n[k], m[k]) for k in range(4)]
    dS = oracle.tucker(T, Ls) - target
    dT, dL = oracle.tucker_adjoint(T, Ls, dS)
    h = 1e-3
    for _ in range(4):
        V = rand(*m)
        fd = (_loss(T + h * V, Ls, target) - _loss(T - h * V, Ls, target)) / (2 * h)
        assert abs(fd - np.sum(dT * V)) <= 1e-9 * max(1.0, abs(fd))
    for mu in range(4):
        V = rand(n[mu], m[mu])
        Lp = list(Ls); Lm = list(Ls)
        Lp[mu] = Ls[mu] + h * V
        Lm[mu] = Ls[mu] - h * V
        fd = (_loss(T, Lp, target) - _loss(T, Lm, target)) / (2 * h)
        assert abs(fd - np.sum(dL[mu] * V)) <= 1e-9 * max(1.0, abs(fd))


def test_adjoint_full_coordinate_fd_tiny():
    m, n = (2, 3, 2), (3, 2, 2)
    T, target = rand(*m), rand(*n)
    Ls = [rand(n[k], m[k]) for k in range(3)]
    dT, dL = oracle.tucker_adjoint(T, Ls, oracle.tucker(T, Ls) - target)
    h = 1e-4
    for idx in np.ndindex(*m):
        E = np.zeros(m, order="F"); E[idx] = 1
        fd = (_loss(T + h * E, Ls, target) - _loss(T - h * E, Ls, target)) / (2 * h)
        assert abs(fd - dT[idx]) <= 1e-8 * max(1.0, abs(fd))
    for mu in range(3):
        for idx in np.ndindex(n[mu], m[mu]):
            E = np.zeros((n[mu], m[mu])); E[idx] = 1
            Lp = list(Ls); Lm = list(Ls)
            Lp[mu] = Ls[mu] + h * E
            Lm[mu] = Ls[mu] - h * E
            fd = (_loss(T, Lp, target) - _loss(T, Lm, target)) / (2 * h)
            assert abs(fd - dL[mu][idx]) <= 1e-8 * max(1.0, abs(fd))


# ----------------------------------------------------------- exponential ---

@pytest.mark.parametrize("n", [1, 2, 5, 12])
def test_expm_closed_form_matches_scipy_and_taylor(n):
    sub, diag, sup = W.fd_advection_diffusion(n)
    t = 1e-4
    A = W.tridiag_dense(n, sub, diag, sup)
    E1 = oracle.expm_tridiag_toeplitz(n, sub, diag, sup, t)
    E2 = oracle.expm_taylor(A, t)
    E3 = scipy.linalg.expm(t * A)
    scale = np.abs(E3).max()
    np.testing.assert_allclose(E1, E3, rtol=0, atol=1e-13 * scale)
    np.testing.assert_allclose(E2, E3, rtol=0, atol=1e-13 * scale)


def test_expm_symmetric_matches_eigendecomposition():
    """a = c: textbook symmetric eigen-decomposition (numpy.linalg.eigh)."""
    n, a, b = 9, 1.3, -2.1
    A = W.tridiag_dense(n, a, b, a)
    lam, V = np.linalg.eigh(A)
    ref = (V * np.exp(0.7 * lam)) @ V.T
    np.testing.assert_allclose(oracle.expm_tridiag_toeplitz(n, a, b, a, 0.7), ref,
                               rtol=0, atol=1e-13)


def test_expm_taylor_nonnormal_small():
    A = rand(6, 6)
    np.testing.assert_allclose(oracle.expm_taylor(A, 0.9), scipy.linalg.expm(0.9 * A),
                               rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("n", [4, 5, 6])
def test_stepper_matches_full_kronecker_sum_expm(n):
    """Eq. (expmat) with the assembled Kronecker sum (exponentiated by the
    long-double Taylor routine) against one step of Eq. (exptucker)."""
    sub, diag, sup = W.fd_advection_diffusion(n)
    tau = 3e-3
    A = W.tridiag_dense(n, sub, diag, sup)
    I = np.eye(n)
    K = np.kron(I, np.kron(I, A)) + np.kron(I, np.kron(A, I)) + np.kron(A, np.kron(I, I))
    U0 = rand(n, n, n)
    ref = oracle.expm_taylor(K, tau) @ oracle.vec(U0)
    E = oracle.expm_tridiag_toeplitz(n, sub, diag, sup, tau)
    U1 = oracle.expkronsum_steps(U0, [E, E, E], 1)
    np.testing.assert_allclose(oracle.vec(U1), ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_stepper_semigroup():
    """k steps with exp(tau A) equal one step with exp(k tau A)."""
    n, k, tau = 7, 5, 2e-3
    sub, diag, sup = W.fd_advection_diffusion(n)
    U0 = rand(n, n, n)
    E1 = oracle.expm_tridiag_toeplitz(n, sub, diag, sup, tau)
    Ek = oracle.expm_tridiag_toeplitz(n, sub, diag, sup, k * tau)
    Uk = oracle.expkronsum_steps(U0, [E1] * 3, k)
    U1 = oracle.expkronsum_steps(U0, [Ek] * 3, 1)
    np.testing.assert_allclose(Uk, U1, rtol=0, atol=1e-12 * np.abs(U1).max())


def test_stepper_pure_diffusion_eigenmode():
    """No advection, a sine eigenmode: pure decay by exp(t sum_mu lambda_mu)."""
    n, tau, steps = 16, 1e-3, 3
    sub, diag, sup = W.fd_advection_diffusion(n, advection=0.0)
    h = 1.0 / (n + 1)
    x = np.arange(1, n + 1) * h
    ks = (1, 2, 3)
    vecs = [np.sin(k * np.pi * x) for k in ks]
    lam = [diag + 2 * sub * np.cos(k * np.pi / (n + 1)) for k in ks]
    U0 = np.asfortranarray(np.multiply.outer(np.multiply.outer(vecs[0], vecs[1]), vecs[2]))
    E = oracle.expm_tridiag_toeplitz(n, sub, diag, sup, tau)
    U = oracle.expkronsum_steps(U0, [E] * 3, steps)
    ref = U0 * np.exp(steps * tau * sum(lam))
    np.testing.assert_allclose(U, ref, rtol=0, atol=1e-13 * np.abs(U0).max())


# --------------------------------------------------- workload matrices ---

def test_chebyshev_vandermonde_discrete_orthogonality():
    n = 20
    L = W.chebyshev_vandermonde(n, n)
    G = L.T @ L
    ref = np.diag([n] + [n / 2] * (n - 1))
    np.testing.assert_allclose(G, ref, rtol=0, atol=1e-12)
    T = rand(n, n, n)
    Dinv = np.diag(1.0 / np.diag(ref))
    back = oracle.mump(oracle.mump(T, L, 1), Dinv @ L.T, 1)
    np.testing.assert_allclose(back, T, rtol=0, atol=1e-12)


@pytest.mark.parametrize("m,n", [(8, 12), (11, 17), (15, 23), (64, 96)])
def test_barycentric_partition_of_unity_and_polynomials(m, n):
    x = W.uniform_points(n)
    L = W.barycentric_matrix(m, x)
    np.testing.assert_allclose(L.sum(axis=1), 1.0, rtol=0, atol=1e-12)
    xi = W.chebyshev_points(m)
    # a separable polynomial of degree < m per direction is reproduced exactly
    c = rand(m)
    p = lambda t: np.polynomial.chebyshev.chebval(t, c)
    F = np.asfortranarray(np.multiply.outer(p(xi), p(xi)))
    P = oracle.tucker(F, [L, L])
    ref = np.multiply.outer(p(x), p(x))
    np.testing.assert_allclose(P, ref, rtol=0, atol=1e-10 * np.abs(ref).max())


def _runge_error(m, n=35):
    xi = W.chebyshev_points(m)
    x = W.uniform_points(n)
    F = W.runge([xi] * 5)
    L = W.barycentric_matrix(m, x)
    P = oracle.tucker(F, [L] * 5)
    return W.rel_err_max(P, W.runge([x] * 5))


def _golden_fig3():
    path = os.path.join(os.path.dirname(__file__), "golden", "fig3_runge_errors.txt")
    rows = []
    for line in open(path):
        line = line.split("#")[0].strip()
        if line:
            m, e = line.split()
            rows.append((int(m), e))
    return rows


@pytest.mark.parametrize("m,printed", [r for r in _golden_fig3() if r[0] <= 25])
def test_runge_interpolation_errors_match_paper(m, printed):
    """Section 4.3, Figure 3: the printed max-norm relative errors, to the
    printed digits."""
    err = _runge_error(m)
    digits = len(printed.split("e")[0].replace(".", "").lstrip("0"))
    ref = float(printed)
    ulp = 10.0 ** (np.floor(np.log10(ref)) - (digits - 1))
    assert abs(err - ref) <= 0.5 * ulp, (m, err, printed)


@pytest.mark.slow
@pytest.mark.parametrize("m,printed", [r for r in _golden_fig3() if r[0] == 35])
def test_runge_interpolation_errors_match_paper_m35(m, printed):
    err = _runge_error(m)
    digits = len(printed.split("e")[0].replace(".", "").lstrip("0"))
    ref = float(printed)
    ulp = 10.0 ** (np.floor(np.log10(ref)) - (digits - 1))
    assert abs(err - ref) <= 0.5 * ulp, (m, err, printed)


# ---------------------------------------------------------------- itucker

def _wc(rng, n):
    """A well-conditioned n x n matrix (I plus a small random part)."""
    return np.eye(n) + 0.3 * rng.standard_normal((n, n)) / np.sqrt(n)


def test_itucker_solves_the_explicit_kronecker_system():
    """vec(S) = (P_3 (x) P_2 (x) P_1)^{-1} vec(V): a dense solve of the
    explicit Kronecker product (Eq. (preconnd) with Lemma "krontomu")."""
    rng = np.random.default_rng(41)
    m = (2, 3, 4)
    V = rng.standard_normal(m)
    Ps = [_wc(rng, n) for n in m]
    K = np.kron(np.kron(Ps[2], Ps[1]), Ps[0])
    ref = np.linalg.solve(K, V.reshape(-1, order="F"))
    S = oracle.itucker(V, Ps)
    np.testing.assert_allclose(S.reshape(-1, order="F"), ref, rtol=0, atol=1e-13 * np.abs(ref).max())


def test_itucker_inverts_the_tucker_operator():
    rng = np.random.default_rng(42)
    m = (5, 7, 3, 4)
    V = rng.standard_normal(m)
    Ps = [_wc(rng, n) for n in m]
    back = oracle.itucker(oracle.tucker(V, Ps), Ps)
    np.testing.assert_allclose(back, V, rtol=0, atol=1e-12 * np.abs(V).max())
    back_t = oracle.itucker(oracle.tucker(V, Ps, transL=True), Ps, transL=True)
    np.testing.assert_allclose(back_t, V, rtol=0, atol=1e-12 * np.abs(V).max())


def test_itucker_identity_and_two_dimensional_case():
    rng = np.random.default_rng(43)
    V = rng.standard_normal((6, 5))
    assert np.array_equal(oracle.itucker(V, [np.eye(6), np.eye(5)]), V)
    P1, P2 = _wc(rng, 6), _wc(rng, 5)
    # d = 2: P_1^{-1} V P_2^{-T} (Section 3.4)
    ref = np.linalg.inv(P1) @ V @ np.linalg.inv(P2).T
    np.testing.assert_allclose(oracle.itucker(V, [P1, P2]), ref, rtol=0, atol=1e-13 * np.abs(ref).max())


# ----------------------------------------------- semilinear IMEX (Section 4.5)

def _golden_table3():
    path = os.path.join(os.path.dirname(__file__), "golden", "table3_semilinear.txt")
    with open(path) as f:
        row = [ln.split() for ln in f if ln.strip() and not ln.startswith("#")][0]
    return tuple(int(v) for v in row[:3]), float(row[3]), float(row[4]), float(row[5]), int(row[6]), int(row[7])


def test_laplacian_eigenpairs_closed_form():
    n = 9
    lam, Q = oracle.laplacian_eig(n)
    A = W.tridiag_dense(n, (n + 1.0) ** 2, -2.0 * (n + 1.0) ** 2, (n + 1.0) ** 2)
    np.testing.assert_allclose(A @ Q, Q * lam, rtol=0, atol=1e-10 * np.abs(lam).max())
    np.testing.assert_allclose(Q.T @ Q, np.eye(n), rtol=0, atol=1e-14)
    np.testing.assert_allclose(np.sort(lam), np.linalg.eigvalsh(A), rtol=1e-13)


def test_kronsum_solve_inverts_the_kronecker_sum():
    """The diagonalised solve against the Kronecker-sum action (Eq. (actkron))
    and a dense solve of the assembled matrix."""
    c = W.semilinear(n=(5, 6, 7), tau=0.01)
    rng = np.random.default_rng(44)
    v = rng.standard_normal(c.n)
    x = oracle.kronsum_solve_laplacian(v, c.n, c.tau)
    np.testing.assert_allclose(oracle.kronsumv(x, c.M), v, rtol=0, atol=1e-13 * np.abs(v).max())
    I = [np.eye(k) for k in c.n]
    Mfull = (np.kron(np.kron(I[2], I[1]), c.M[0]) + np.kron(np.kron(I[2], c.M[1]), I[0])
             + np.kron(np.kron(c.M[2], I[1]), I[0]))
    ref = np.linalg.solve(Mfull, v.reshape(-1, order="F"))
    np.testing.assert_allclose(x.reshape(-1, order="F"), ref, rtol=0, atol=1e-13 * np.abs(ref).max())


def test_semilinear_final_error_matches_the_paper():
    """Section 4.5: final relative error 9.7e-3 at n = (40, 44, 48), tau = 0.01,
    t* = 1.  The scheme with exact solves gives 9.76e-3, which agrees with the
    printed two digits when the printed value is truncated; accepted band
    [9.6e-3, 9.8e-3]."""
    n, tau, tstar, printed, _, _ = _golden_table3()
    c = W.semilinear(n=n, tau=tau, tstar=tstar)
    u = oracle.semilinear_imex(c)
    ex = c.exact(tstar)
    err = np.abs(u - ex).max() / np.abs(ex).max()
    assert abs(err - printed) <= 0.1e-3, err
    assert err == pytest.approx(9.7576e-3, rel=1e-3)


# ------------------------------------------------------------------ complex

def _crand(*shape, seed=0):
    g = np.random.default_rng(2112 + seed)
    return np.asfortranarray(g.standard_normal(shape) + 1j * g.standard_normal(shape))


def test_ctucker_on_real_inputs_equals_the_real_oracle():
    """Over real data the complex operator is the real one (C oracle, Eq. (tuckerop))."""
    g = np.random.default_rng(5)
    T = g.standard_normal((4, 5, 3))
    Ls = [g.standard_normal((6, 4)), g.standard_normal((2, 5)), g.standard_normal((3, 3))]
    S = oracle.ctucker(T, Ls)
    assert np.max(np.abs(S.imag)) == 0.0
    assert np.allclose(S.real, oracle.tucker(T, Ls), rtol=0, atol=1e-13)
    Lt = [np.asfortranarray(L.T) for L in Ls]
    assert np.allclose(oracle.ctucker(T, Lt, transL=True).real, oracle.tucker(T, Lt, transL=True),
                       rtol=0, atol=1e-13)


@pytest.mark.parametrize("transL,conj", [(False, False), (True, False), (True, True), (False, True)])
def test_ctucker_equals_nested_sum(transL, conj):
    """Brute force over C of Eq. (nestedmumode)."""
    T = _crand(3, 2, 4, seed=1)
    shapes = [(2, 3), (3, 2), (4, 4)]
    Ls = [_crand(*(s[::-1] if transL else s), seed=2 + k) for k, s in enumerate(shapes)]
    ref = oracle.ctucker_nested(T, Ls, transL, conj)
    assert np.allclose(oracle.ctucker(T, Ls, transL, conj), ref, rtol=0, atol=1e-12)


def test_cttucker_with_dft_matrices_is_the_inverse_fft():
    """Psi_mu = F (the DFT matrix, F[j, k] = exp(-2 pi i j k / m)): T x_mu F is
    numpy.fft.fftn, and the conjugate transposes (cttucker) give m_1...m_d
    times numpy.fft.ifftn (a library routine, independent of the oracle)."""
    T = _crand(8, 5, 6, seed=7)
    Fs = [np.exp(-2j * np.pi * np.outer(np.arange(m), np.arange(m)) / m) for m in T.shape]
    assert np.allclose(oracle.ctucker(T, Fs), np.fft.fftn(T), rtol=0, atol=1e-10)
    assert np.allclose(oracle.ctucker(T, Fs, transL=True, conj=True), np.fft.ifftn(T) * T.size, rtol=0, atol=1e-10)


def test_cttucker_with_unitary_matrices_keeps_the_norm():
    """Unitary Psi_mu: the operator with the conjugate transposes is the inverse
    of the one with Psi_mu, and both keep the Frobenius norm."""
    T = _crand(5, 4, 6, seed=9)
    Us = [np.linalg.qr(_crand(m, m, seed=20 + m))[0] for m in T.shape]
    S = oracle.ctucker(T, Us, transL=True, conj=True)
    assert np.isclose(np.linalg.norm(S), np.linalg.norm(T), rtol=1e-13)
    assert np.allclose(oracle.ctucker(S, Us), T, rtol=0, atol=1e-12)


def test_ctucker_conjugation_identity():
    """conj(T x op(L)^*) = conj(T) x op(L) elementwise (complex conjugation is a ring automorphism)."""
    T = _crand(3, 4, seed=11)
    Ls = [_crand(3, 5, seed=12), _crand(4, 2, seed=13)]
    a = oracle.ctucker(T, Ls, transL=True, conj=True)
    b = oracle.ctucker(T.conj(), Ls, transL=True, conj=False).conj()
    assert np.allclose(a, b, rtol=0, atol=1e-13)


# ------------------------------------------------- Hermite--Laguerre--Fourier

def _golden_hlf():
    rows = []
    with open(os.path.join(os.path.dirname(__file__), "golden", "fig_spectral_hlf_accuracy.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                m1, m2, m3, acc = line.split()
                rows.append(((int(m1), int(m2), int(m3)), float(acc)))
    return rows


@pytest.mark.parametrize("m,beta", [(1, 1.0), (7, 0.7), (45, 1.7), (69, 2.1)])
def test_hermite_rule_makes_the_functions_orthonormal(m, beta):
    """Gauss exactness: Psi diag(w) Psi^T = I for the m functions at the m nodes
    (every product H_i H_j, i, j < m, is integrated exactly)."""
    x, w = oracle.gauss_hermite(m, beta)
    Psi = oracle.hermite_functions(m, beta, x).T
    assert np.allclose(Psi @ np.diag(w) @ Psi.T, np.eye(m), rtol=0, atol=1e-12)


@pytest.mark.parametrize("m,alpha,beta", [(1, 4.0, 1.0), (6, 0.0, 1.3), (31, 4.0, 12.3), (60, 1.5, 0.8)])
def test_laguerre_rule_makes_the_functions_orthonormal(m, alpha, beta):
    x, w = oracle.gauss_laguerre(m, alpha, beta)
    Psi = oracle.laguerre_functions(m, alpha, beta, x).T
    assert np.allclose(Psi @ np.diag(w) @ Psi.T, np.eye(m), rtol=0, atol=1e-11)


def test_hermite_and_laguerre_functions_match_the_closed_forms():
    """Against scipy's Hermite and generalized Laguerre polynomials with the
    normalisations of the paper's definitions (low degrees)."""
    import math
    import scipy.special as sp
    x = np.linspace(-3, 3, 41)
    beta = 1.3
    H = oracle.hermite_functions(9, beta, x)
    for i in range(9):
        ref = np.sqrt(beta / (np.sqrt(np.pi) * 2.0 ** i * math.factorial(i))) * sp.eval_hermite(i, beta * x) \
            * np.exp(-(beta * x) ** 2 / 2)
        assert np.allclose(H[:, i], ref, rtol=1e-12, atol=1e-14)
    x = np.linspace(0, 9, 37)
    alpha, beta = 4.0, 0.9
    Lg = oracle.laguerre_functions(9, alpha, beta, x)
    for i in range(9):
        ref = np.sqrt(beta * math.factorial(i) / math.gamma(i + alpha + 1)) * sp.eval_genlaguerre(i, alpha, beta * x) \
            * (beta * x) ** (alpha / 2) * np.exp(-beta * x / 2)
        assert np.allclose(Lg[:, i], ref, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("m,n", [(8, 301), (7, 20), (38, 301), (1, 5)])
def test_fourier_resample_reproduces_trigonometric_polynomials(m, n):
    """The resampling of the samples of any trigonometric polynomial of degree
    below m/2 equals its values at the new points; constants stay constant."""
    F = oracle.fourier_resample(m, n)
    assert np.allclose(F.sum(axis=1), 1.0, atol=1e-13)
    t, s = np.arange(m) / m, np.arange(n) / n
    for k in range(1, (m + 1) // 2):
        for fn in (np.sin, np.cos):
            assert np.allclose(F @ fn(2 * np.pi * k * t), fn(2 * np.pi * k * s), atol=1e-12)


@pytest.mark.parametrize("m", [1, 2, 7, 8, 64])
def test_fourier_resample_interpolates_the_samples(m):
    """At the sample points themselves (n = m) the interpolant reproduces the
    samples: the matrix is the identity, odd and even m alike."""
    assert np.allclose(oracle.fourier_resample(m, m), np.eye(m), rtol=0, atol=1e-13)


def test_hlf_decomposition_reproduces_the_paper():
    """The HLF experiment through the oracle's Tucker operator reproduces the
    accuracies the paper plots for (m1, m2, m3) = (45, 31, 8) ... (69, 105, 38)."""
    for (m1, m2, m3), acc in _golden_hlf():
        err = oracle.hlf_error(m1, m2, m3)
        assert abs(err - acc) <= 2e-3 * acc, ((m1, m2, m3), err, acc)
