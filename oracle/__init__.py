"""FP64 CPU oracle for the mu-mode product, the Tucker operator and what they drive.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library and never imports it.

Tensors are numpy arrays of any memory order; they are handed to the C code
column-major (Fortran order), the layout of the vec operator of Appendix A.
A matrix ``L`` of shape ``(n, m)`` acts on fibres of length ``m``.

The C source is ``kron_oracle.c`` next to this file; it is compiled on first
use (gcc, -O2, OpenMP, no fast-math, no FP contraction) into
``libkron_oracle.so``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kron_oracle.c")
_LIB = os.path.join(_HERE, "libkron_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle into a shared library next to the source."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp.%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(_LIB)
        i64p = ctypes.POINTER(ctypes.c_int64)
        dp = ctypes.c_void_p
        _lib.oracle_mump.argtypes = [ctypes.c_int, i64p, ctypes.c_int, ctypes.c_int64, dp, dp,
                                     ctypes.c_int64, ctypes.c_int, dp]
        _lib.oracle_tucker.argtypes = [ctypes.c_int, i64p, i64p, dp, dp, i64p, ctypes.c_int, dp]
        _lib.oracle_tucker_nested.argtypes = [ctypes.c_int, i64p, i64p, dp, dp, i64p, ctypes.c_int, dp]
        _lib.oracle_kron.argtypes = [ctypes.c_int64, ctypes.c_int64, dp, ctypes.c_int64,
                                     ctypes.c_int64, dp, dp]
        _lib.oracle_matvec.argtypes = [ctypes.c_int64, ctypes.c_int64, dp, dp, dp]
        _lib.oracle_tucker_adjoint.argtypes = [ctypes.c_int, i64p, i64p, dp, dp, i64p, dp, dp, dp]
        _lib.oracle_expm_tridiag_toeplitz.argtypes = [ctypes.c_int64, ctypes.c_double,
                                                      ctypes.c_double, ctypes.c_double,
                                                      ctypes.c_double, dp]
        _lib.oracle_expm_taylor.argtypes = [ctypes.c_int64, dp, ctypes.c_double, dp]
        _lib.oracle_expkronsum_steps.argtypes = [ctypes.c_int, i64p, dp, ctypes.c_int, dp]
        _lib.oracle_kronsumv.argtypes = [ctypes.c_int, i64p, dp, dp, i64p, dp]
        _lib.oracle_num_threads.restype = ctypes.c_int
    return _lib


def num_threads() -> int:
    """OpenMP threads the oracle uses (the host cores it runs on)."""
    return int(_load().oracle_num_threads())


def _f64(a) -> np.ndarray:
    return np.asfortranarray(np.asarray(a, dtype=np.float64))


def _i64(vals) -> ctypes.Array:
    arr = (ctypes.c_int64 * len(vals))(*[int(v) for v in vals])
    return arr


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def mump(T, L, mu: int, transL: bool = False) -> np.ndarray:
    """``T x_mu op(L)`` (Eq. (mmp)); ``mu`` is 0-based.  op(L) = L, or L^T if transL."""
    T = _f64(T)
    L = _f64(L)
    m = list(T.shape)
    d = len(m)
    n = L.shape[1] if transL else L.shape[0]
    out = list(m)
    out[mu] = n
    S = np.zeros(out, dtype=np.float64, order="F")
    ld = max(L.shape[0], 1)
    _check(_load().oracle_mump(d, _i64(m), mu, n, _ptr(T), _ptr(L), ld, int(transL), _ptr(S)), "mump")
    return S


def _mat_table(Ls):
    Ls = [_f64(L) for L in Ls]
    ptrs = (ctypes.c_void_p * len(Ls))(*[_ptr(L) for L in Ls])
    lds = _i64([max(L.shape[0], 1) for L in Ls])
    return Ls, ptrs, lds


def tucker(T, Ls, transL: bool = False) -> np.ndarray:
    """Tucker operator ``T x_1 op(L_1) ... x_d op(L_d)`` (Eq. (tuckerop)), modes in order 1..d."""
    T = _f64(T)
    m = list(T.shape)
    d = len(m)
    Ls, ptrs, lds = _mat_table(Ls)
    n = [(L.shape[1] if transL else L.shape[0]) for L in Ls]
    S = np.zeros(n, dtype=np.float64, order="F")
    _check(_load().oracle_tucker(d, _i64(m), _i64(n), _ptr(T), ptrs, lds, int(transL), _ptr(S)),
           "tucker")
    return S


def tucker_nested(T, Ls, transL: bool = False) -> np.ndarray:
    """Brute-force element-wise sum of Eq. (nestedmumode); tiny inputs only."""
    T = _f64(T)
    m = list(T.shape)
    d = len(m)
    Ls, ptrs, lds = _mat_table(Ls)
    n = [(L.shape[1] if transL else L.shape[0]) for L in Ls]
    S = np.zeros(n, dtype=np.float64, order="F")
    _check(_load().oracle_tucker_nested(d, _i64(m), _i64(n), _ptr(T), ptrs, lds, int(transL),
                                        _ptr(S)), "tucker_nested")
    return S


def kron(A, B) -> np.ndarray:
    """Kronecker product ``A (x) B`` as defined in Appendix A."""
    A = _f64(np.atleast_2d(A))
    B = _f64(np.atleast_2d(B))
    C = np.zeros((A.shape[0] * B.shape[0], A.shape[1] * B.shape[1]), order="F")
    _check(_load().oracle_kron(A.shape[0], A.shape[1], _ptr(A), B.shape[0], B.shape[1], _ptr(B),
                               _ptr(C)), "kron")
    return C


def matvec(A, x) -> np.ndarray:
    A = _f64(A)
    x = _f64(np.ravel(x, order="F"))
    y = np.zeros(A.shape[0])
    _check(_load().oracle_matvec(A.shape[0], A.shape[1], _ptr(A), _ptr(x), _ptr(y)), "matvec")
    return y


def vec(T) -> np.ndarray:
    """vec operator of Appendix A: first index fastest."""
    return np.ravel(np.asarray(T), order="F")


def tucker_adjoint(T, Ls, dS, want_dT: bool = True, want_dL: bool = True):
    """Gradients of <S, dS> with S = tucker(T, Ls): returns (dT, [dL_mu])."""
    T = _f64(T)
    dS = _f64(dS)
    m = list(T.shape)
    d = len(m)
    Ls, ptrs, lds = _mat_table(Ls)
    n = [L.shape[0] for L in Ls]
    dT = np.zeros(m, order="F") if want_dT else None
    dL = [np.zeros((n[k], m[k]), order="F") for k in range(d)] if want_dL else None
    dLp = (ctypes.c_void_p * d)(*[_ptr(x) for x in dL]) if want_dL else None
    _check(_load().oracle_tucker_adjoint(d, _i64(m), _i64(n), _ptr(T), ptrs, lds, _ptr(dS),
                                         _ptr(dT) if want_dT else None, dLp), "tucker_adjoint")
    return dT, dL


def expm_tridiag_toeplitz(n: int, a: float, b: float, c: float, t: float) -> np.ndarray:
    """Closed-form exp(t A) for A = tridiag(a, b, c) (sub, diag, super), long double inside."""
    E = np.zeros((n, n), order="F")
    _check(_load().oracle_expm_tridiag_toeplitz(n, a, b, c, t, _ptr(E)), "expm_tridiag_toeplitz")
    return E


def expm_taylor(A, t: float = 1.0) -> np.ndarray:
    """exp(t A) by long-double Taylor series with scaling and squaring (small A only)."""
    A = _f64(A)
    n = A.shape[0]
    E = np.zeros((n, n), order="F")
    _check(_load().oracle_expm_taylor(n, _ptr(A), t, _ptr(E)), "expm_taylor")
    return E


def expkronsum_steps(U0, Es, nsteps: int) -> np.ndarray:
    """nsteps steps U <- U x_1 E_1 ... x_d E_d (Eq. (exptucker)); returns a new array."""
    U = np.array(_f64(U0), order="F", copy=True)
    n = list(U.shape)
    d = len(n)
    Es = [_f64(E) for E in Es]
    ptrs = (ctypes.c_void_p * d)(*[_ptr(E) for E in Es])
    _check(_load().oracle_expkronsum_steps(d, _i64(n), ptrs, nsteps, _ptr(U)), "expkronsum_steps")
    return U


def kronsumv(V, Ls) -> np.ndarray:
    """Action of the Kronecker sum, Eq. (actkron): sum_mu V x_mu L_mu."""
    V = _f64(V)
    n = list(V.shape)
    d = len(n)
    Ls, ptrs, lds = _mat_table(Ls)
    S = np.zeros(n, order="F")
    _check(_load().oracle_kronsumv(d, _i64(n), _ptr(V), ptrs, lds, _ptr(S)), "kronsumv")
    return S


def ctucker(T, Ls, transL: bool = False, conj: bool = False) -> np.ndarray:
    """Complex Tucker operator T x_1 op(L_1) ... x_d op(L_d) (Eq. (tuckerop) over C),
    op(L) = L, L^T (transL) or the conjugate of either (conj); transL with conj
    is the conjugate transpose of the remark after Eq. (tensinterp) (cttucker).

    Mode by mode in the order 1..d, each mu-mode product by its definition
    S^{(mu)} = op(L_mu) X^{(mu)} (Eq. (mmp)) on the mu-unfolding, in complex128
    (numpy.tensordot as the matrix product)."""
    X = np.array(T, dtype=np.complex128)
    for mu in range(X.ndim):
        G = np.asarray(Ls[mu], dtype=np.complex128)
        if transL:
            G = G.T
        if conj:
            G = G.conj()
        X = np.moveaxis(np.tensordot(G, X, axes=([1], [mu])), 0, mu)
    return np.asfortranarray(X)


def ctucker_nested(T, Ls, transL: bool = False, conj: bool = False) -> np.ndarray:
    """Brute-force element-wise sum of Eq. (nestedmumode) over C (tiny inputs):
    S[l_1..l_d] = sum_{i_1..i_d} T[i_1..i_d] prod_mu op(L_mu)[l_mu, i_mu]."""
    import itertools
    T = np.asarray(T, dtype=np.complex128)
    Gs = []
    for L in Ls:
        G = np.asarray(L, dtype=np.complex128)
        G = G.T if transL else G
        Gs.append(G.conj() if conj else G)
    n = [G.shape[0] for G in Gs]
    S = np.zeros(n, dtype=np.complex128)
    for l in itertools.product(*[range(v) for v in n]):
        acc = 0j
        for i in itertools.product(*[range(v) for v in T.shape]):
            w = T[i]
            for mu in range(T.ndim):
                w = w * Gs[mu][l[mu], i[mu]]
            acc += w
        S[l] = acc
    return S


# ------------------------------------------------ Hermite--Laguerre--Fourier
# The pseudospectral example of Section "Hermite--Laguerre--Fourier function
# decomposition": the functions are the paper's normalized and scaled ones
# with 0-based index i (the paper's i_mu - 1).


def hermite_functions(m: int, beta: float, x) -> np.ndarray:
    """n x m matrix of the normalized scaled Hermite functions
    H_i(x) = sqrt(beta / (sqrt(pi) 2^i i!)) H_i(beta x) exp(-beta^2 x^2 / 2),
    by the recurrence of the orthonormal functions (plain float64; moderate
    m and |x| only)."""
    y = beta * np.asarray(x, dtype=np.float64).ravel()
    F = np.zeros((y.size, m))
    F[:, 0] = np.sqrt(beta) * np.pi ** -0.25 * np.exp(-y * y / 2)
    if m > 1:
        F[:, 1] = np.sqrt(2.0) * y * F[:, 0]
    for i in range(2, m):
        F[:, i] = np.sqrt(2.0 / i) * y * F[:, i - 1] - np.sqrt((i - 1) / i) * F[:, i - 2]
    return F


def laguerre_functions(m: int, alpha: float, beta: float, x) -> np.ndarray:
    """n x m matrix of the normalized scaled generalized Laguerre functions
    L_i(x) = sqrt(beta i! / Gamma(i + alpha + 1)) L_i^alpha(beta x) (beta x)^(alpha/2) exp(-beta x / 2),
    by the recurrence of the orthonormal functions (plain float64)."""
    import math
    y = beta * np.asarray(x, dtype=np.float64).ravel()
    F = np.zeros((y.size, m))
    F[:, 0] = np.sqrt(beta / math.gamma(alpha + 1)) * y ** (alpha / 2) * np.exp(-y / 2)
    if m > 1:
        F[:, 1] = (alpha + 1 - y) / np.sqrt(alpha + 1) * F[:, 0]
    for i in range(2, m):
        F[:, i] = ((2 * i - 1 + alpha - y) * F[:, i - 1] - np.sqrt((i - 1) * (i - 1 + alpha)) * F[:, i - 2]) \
            / np.sqrt(i * (i + alpha))
    return F


def gauss_hermite(m: int, beta: float):
    """Scaled Gauss--Hermite nodes x = xi / beta and function weights
    w = lambda exp(xi^2) / beta (lambda the weights of exp(-xi^2));
    numpy.polynomial.hermite.hermgauss as the rule."""
    from numpy.polynomial.hermite import hermgauss
    xi, lam = hermgauss(m)
    return xi / beta, lam * np.exp(xi * xi) / beta


def gauss_laguerre(m: int, alpha: float, beta: float):
    """Scaled generalized Gauss--Laguerre nodes and function weights
    w = lambda exp(xi) xi^(-alpha) / beta; scipy.special.roots_genlaguerre as the rule."""
    import scipy.special
    xi, lam = scipy.special.roots_genlaguerre(m, alpha)
    return xi / beta, lam * np.exp(xi) * xi ** (-alpha) / beta


def fourier_resample(m: int, n: int) -> np.ndarray:
    """Real n x m matrix (n >= m) of the FFT resampling of m equispaced samples
    of one period to n equispaced points: the spectrum of the samples is
    zero-padded to length n (for n > m the even-m Nyquist coefficient split
    between +-m/2; for n = m the two are one bin and the spectrum is kept
    whole) and transformed back, scaled by n / m."""
    if n < m:
        raise ValueError("the zero-padding resampling needs n >= m")
    F = np.zeros((n, m))
    h = (m + 1) // 2
    for j in range(m):
        e = np.zeros(m)
        e[j] = 1.0
        a = np.fft.fft(e)
        b = np.zeros(n, dtype=np.complex128)
        b[:h] = a[:h]
        b[n - (m - h):] = a[h:]
        if m % 2 == 0 and n > m:
            b[h] = a[h] / 2
            b[n - h] = a[h] / 2
        F[:, j] = np.real(np.fft.ifft(b)) * n / m
    return F


def hlf_function(x1, x2, x3):
    """The trivariate test function of the HLF example."""
    return x2 ** 2 * np.sin(20 * x1) * np.sin(10 * x2) * np.exp(-x1 ** 2 - 2 * x2) / (np.sin(2 * np.pi * x3) + 2)


def hlf_error(m1: int, m2: int, m3: int, alpha: float = 4.0, b1: float = 4.0, b2: float = 11.0,
              a3: float = -1.0, b3: float = 1.0, n: int = 301) -> float:
    """Achieved accuracy of the HLF decomposition with (m1, m2, m3) basis
    functions: coefficients Fhat = FW x_1 Psi_1 x_2 Psi_2 (FW the function at
    the quadrature points times the weights, Psi_mu the functions at the
    nodes), evaluation Ftilde = Fhat x_1 Phi_1 x_2 Phi_2 x_3 Phi_3 (Phi_3 the
    Fourier resampling), both by the Tucker operator (Eq. (tensinterp)), on n
    equispaced points per direction (left end included, right end excluded);
    max-norm relative error against f.  beta_1 = sqrt(2 m1 + 1) / b1,
    beta_2 = (4 m2 + 2 alpha + 2) / b2."""
    beta1 = np.sqrt(2 * m1 + 1) / b1
    beta2 = (4 * m2 + 2 * alpha + 2) / b2
    xi1, w1 = gauss_hermite(m1, beta1)
    xi2, w2 = gauss_laguerre(m2, alpha, beta2)
    xi3 = a3 + (b3 - a3) * np.arange(m3) / m3
    FW = hlf_function(xi1[:, None, None], xi2[None, :, None], xi3[None, None, :]) \
        * w1[:, None, None] * w2[None, :, None]
    Psi1 = hermite_functions(m1, beta1, xi1).T
    Psi2 = laguerre_functions(m2, alpha, beta2, xi2).T
    Fhat = tucker(FW, [Psi1, Psi2, np.eye(m3)])
    x1 = -b1 + 2 * b1 * np.arange(n) / n
    x2 = b2 * np.arange(n) / n
    x3 = a3 + (b3 - a3) * np.arange(n) / n
    Ft = tucker(Fhat, [hermite_functions(m1, beta1, x1), laguerre_functions(m2, alpha, beta2, x2),
                       fourier_resample(m3, n)])
    F = hlf_function(x1[:, None, None], x2[None, :, None], x3[None, None, :])
    return float(np.max(np.abs(Ft - F)) / np.max(np.abs(F)))


def itucker(V, Ps, transL: bool = False) -> np.ndarray:
    """V x_1 op(P_1)^{-1} x_2 ... x_d op(P_d)^{-1} (Section 3.4, Eq. (preconnd)).

    Mode by mode in the order 1..d: the mu-mode product with op(P_mu)^{-1} is
    the solution X^{(mu)} of op(P_mu) X^{(mu)} = current^{(mu)} on the
    mu-unfolding (Eq. (mmp)), by LU with partial pivoting (numpy.linalg.solve,
    LAPACK gesv); no inverse is formed."""
    X = np.array(V, dtype=np.float64)
    for mu in range(X.ndim):
        P = np.asarray(Ps[mu], dtype=np.float64)
        A = P.T if transL else P
        Xm = np.moveaxis(X, mu, 0)
        shape = Xm.shape
        Y = np.linalg.solve(A, Xm.reshape(shape[0], -1))
        X = np.moveaxis(Y.reshape(shape), 0, mu)
    return np.asfortranarray(X)


def laplacian_eig(n: int):
    """Eigenpairs of tridiag(1, -2, 1) / h^2, h = 1/(n+1) (textbook closed
    form): lambda_k = -4 / h^2 sin^2(k pi / (2 (n + 1))), orthonormal
    eigenvectors Q_jk = sqrt(2 / (n + 1)) sin(j k pi / (n + 1)), j, k = 1..n."""
    k = np.arange(1, n + 1)
    h = 1.0 / (n + 1)
    lam = -4.0 / h ** 2 * np.sin(k * np.pi / (2.0 * (n + 1))) ** 2
    Q = np.sqrt(2.0 / (n + 1)) * np.sin(np.outer(k, k) * np.pi / (n + 1))
    return lam, np.asfortranarray(Q)


def kronsum_solve_laplacian(V, n, tau: float):
    """x with (M_d (+) ... (+) M_1) x = v, M_mu = I/d - tau A_mu, A_mu the FD
    Laplacians: exact (up to rounding) by diagonalisation, x = Q D^{-1} Q^T v
    with Q = Q_d (x) ... (x) Q_1 applied as Tucker operators and
    D = 1 - tau (lambda_d (+) ... (+) lambda_1)."""
    eig = [laplacian_eig(k) for k in n]
    W = tucker(V, [Q.T.copy(order="F") for _, Q in eig])
    D = np.ones(tuple(n))
    for mu, (lam, _) in enumerate(eig):
        shape = [1] * len(n)
        shape[mu] = n[mu]
        D = D - tau * lam.reshape(shape)
    return tucker(np.asfortranarray(W / D), [Q for _, Q in eig])


def semilinear_imex(case) -> np.ndarray:
    """Backward-forward (IMEX) Euler of Section 4.5, Eq. (semilin-disc):
    M u_{k+1} = u_k + tau f(t_k, u_k), f = 1 / (1 + u^2) + Phi(t_k, x),
    M = M_3 (+) M_2 (+) M_1, every system solved exactly
    (kronsum_solve_laplacian).  Returns u at t* = nsteps tau."""
    u = np.array(case.U0, order="F")
    for k in range(case.nsteps):
        t = k * case.tau
        rhs = u + case.tau * (1.0 / (1.0 + u ** 2) + case.phi(t))
        u = kronsum_solve_laplacian(rhs, case.n, case.tau)
    return u
