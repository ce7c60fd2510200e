"""Seeded synthetic inputs for the Tucker-operator workloads.

This module only *generates inputs*: random tensors, the interpolation and
transform matrices L_mu that the workloads feed to the Tucker operator, the
finite-difference matrices A_mu of the stepper, and the initial field.  It
holds none of the mu-mode / Tucker / exponential arithmetic; both the FP64
oracle and the GPU path take their inputs from here.

All arrays are numpy float64 in Fortran (column-major) order, the layout of
the vec operator of Appendix A.  Randomness comes from numpy's PCG64 seeded
with ``(seed, object_id)`` so that every object of a workload has its own
independent, reproducible stream.

Workloads (sizes are the ones the benchmark and the parity tests use):

* ``tucker_d3``     : d = 3, n = m = 100, T and L_mu standard normal.
* ``stepper``       : d = 3, n = 256, A_mu = FD Laplacian on [0, 1]
                      (Dirichlet) plus centred advection 0.5, tau = 1e-4,
                      100 steps, smooth rank-4 initial field.
* ``tucker_d6``     : d = 6, n = m = 20, T standard normal, L_mu
                      Chebyshev-Vandermonde matrices cos(k arccos x_i).
* ``batched``       : 512 tensors, d = 3, m_mu uniform in [8, 64],
                      n_mu = ceil(1.5 m_mu), L_mu barycentric Lagrange
                      matrices from Chebyshev points to uniform points.
* ``adjoint``       : d = 4, n = m = 48, T, L_mu, S_target standard normal.
* ``semilinear``    : the 3-D semilinear problem of Section 4.5, n = (40, 44,
                      48) interior points, tau = 0.01, t* = 1: FD Laplacians,
                      the IMEX factors M_mu = I/3 - tau A_mu and the ADI
                      factors P_mu = I - tau A_mu, u_0, and the forcing Phi
                      that makes e^t u_0 the exact solution.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def rng(seed: int, obj: int = 0) -> np.random.Generator:
    """Independent PCG64 stream for object ``obj`` of a workload seeded by ``seed``."""
    return np.random.default_rng([int(seed), int(obj)])


def normal(shape, seed: int, obj: int = 0) -> np.ndarray:
    """i.i.d. standard normal array (Fortran order)."""
    g = rng(seed, obj)
    n = int(np.prod(shape)) if len(shape) else 1
    return np.asfortranarray(g.standard_normal(n).reshape(shape, order="F"))


# --------------------------------------------------------------------------
# 1-D rules used as the L_mu of the interpolation / transform workloads
# --------------------------------------------------------------------------

def chebyshev_points(m: int) -> np.ndarray:
    """First-kind Chebyshev nodes xi_k = cos((2k-1) pi / (2m)), k = 1..m.

    Evaluated as sin(pi (m - 2k + 1) / (2m)) (the same value), which is exactly
    antisymmetric and gives an exact 0 for the middle node of odd m.
    """
    k = np.arange(1, m + 1, dtype=np.float64)
    return np.sin(np.pi * (m - 2.0 * k + 1.0) / (2.0 * m))


def chebyshev_weights(m: int) -> np.ndarray:
    """Barycentric weights of the first-kind nodes: (-1)^(k+1) sin((2k-1) pi / (2m))."""
    k = np.arange(1, m + 1, dtype=np.float64)
    return ((-1.0) ** (k + 1)) * np.sin((2.0 * k - 1.0) * np.pi / (2.0 * m))


def uniform_points(n: int) -> np.ndarray:
    """n uniformly spaced points on [-1, 1], endpoints included."""
    if n == 1:
        return np.zeros(1)
    return -1.0 + 2.0 * np.arange(n, dtype=np.float64) / (n - 1)


def barycentric_matrix(m: int, x: np.ndarray) -> np.ndarray:
    """Lagrange basis of the m Chebyshev nodes evaluated at x, in the second
    barycentric form: L[l, k] = (w_k / (x_l - xi_k)) / sum_j w_j / (x_l - xi_j).
    A point that coincides with a node gets the unit row e_k."""
    xi = chebyshev_points(m)
    w = chebyshev_weights(m)
    x = np.asarray(x, dtype=np.float64)
    L = np.zeros((x.size, m))
    for l, xl in enumerate(x):
        diff = xl - xi
        hit = np.nonzero(diff == 0.0)[0]
        if hit.size:
            L[l, hit[0]] = 1.0
            continue
        r = w / diff
        L[l, :] = r / r.sum()
    return np.asfortranarray(L)


def chebyshev_vandermonde(n: int, m: int) -> np.ndarray:
    """L[i, k] = cos(k arccos x_i) = T_k(x_i) at the n first-kind Chebyshev
    points x_i = cos((2i-1) pi / (2n)), degrees k = 0..m-1."""
    theta = (2.0 * np.arange(1, n + 1) - 1.0) * np.pi / (2.0 * n)
    k = np.arange(m, dtype=np.float64)
    return np.asfortranarray(np.cos(np.outer(theta, k)))


# --------------------------------------------------------------------------
# Stepper inputs
# --------------------------------------------------------------------------

def fd_advection_diffusion(n: int, advection: float = 0.5):
    """Tridiagonal coefficients (sub, diag, super) of A = D2 - advection * D1 on
    the n interior points of [0, 1] with Dirichlet ends, h = 1/(n+1):
    D2 = tridiag(1, -2, 1) / h^2, D1 = tridiag(-1, 0, 1) / (2h)."""
    h = 1.0 / (n + 1)
    sub = 1.0 / h ** 2 + advection / (2.0 * h)
    diag = -2.0 / h ** 2
    sup = 1.0 / h ** 2 - advection / (2.0 * h)
    return sub, diag, sup


def tridiag_dense(n: int, sub: float, diag: float, sup: float) -> np.ndarray:
    A = np.zeros((n, n), order="F")
    idx = np.arange(n)
    A[idx, idx] = diag
    A[idx[1:], idx[:-1]] = sub
    A[idx[:-1], idx[1:]] = sup
    return A


def smooth_field_factors(n: int, d: int, rank: int, seed: int, nmodes: int = 8):
    """Factors f_{r,mu}(x_j) = sum_{k=1..nmodes} g_{r,mu,k} sin(k pi x_j) / k^2 on
    the interior grid x_j = j/(n+1), g standard normal.  Returns an array of
    shape (rank, d, n)."""
    g = rng(seed, 7).standard_normal((rank, d, nmodes))
    x = np.arange(1, n + 1, dtype=np.float64) / (n + 1)
    k = np.arange(1, nmodes + 1, dtype=np.float64)
    basis = np.sin(np.pi * np.outer(k, x)) / (k[:, None] ** 2)       # (nmodes, n)
    return np.einsum("rdk,kn->rdn", g, basis)


def outer_sum(factors: np.ndarray) -> np.ndarray:
    """sum_r f_{r,1} o f_{r,2} o ... o f_{r,d} as a Fortran-ordered tensor."""
    rank, d, n = factors.shape
    U = None
    for r in range(rank):
        t = factors[r, 0]
        for mu in range(1, d):
            t = np.multiply.outer(t, factors[r, mu])
        U = t if U is None else U + t
    return np.asfortranarray(U)


# --------------------------------------------------------------------------
# Workload descriptions
# --------------------------------------------------------------------------

@dataclass
class TuckerCase:
    T: np.ndarray
    L: list
    name: str = ""


@dataclass
class StepperCase:
    n: int
    d: int
    tau: float
    nsteps: int
    tri: tuple            # (sub, diag, super) of every A_mu
    A: list               # dense A_mu
    factors: np.ndarray   # (rank, d, n) factors of U_0
    U0: np.ndarray | None = None


@dataclass
class BatchedCase:
    m: np.ndarray         # (batch, d) int
    n: np.ndarray         # (batch, d) int
    T: list = field(default_factory=list)
    L: list = field(default_factory=list)   # list of lists


SEED = 2112


def tucker_d3(n: int = 100, seed: int = SEED + 1) -> TuckerCase:
    T = normal((n, n, n), seed, 0)
    L = [normal((n, n), seed, 1 + k) for k in range(3)]
    return TuckerCase(T, L, f"tucker d=3 n=m={n} fp64")


def stepper(n: int = 256, d: int = 3, tau: float = 1e-4, nsteps: int = 100,
            seed: int = SEED + 2, rank: int = 4, with_u0: bool = True) -> StepperCase:
    tri = fd_advection_diffusion(n)
    A = [tridiag_dense(n, *tri) for _ in range(d)]
    f = smooth_field_factors(n, d, rank, seed)
    U0 = outer_sum(f) if with_u0 else None
    return StepperCase(n, d, tau, nsteps, tri, A, f, U0)


def tucker_d6(n: int = 20, d: int = 6, seed: int = SEED + 3) -> TuckerCase:
    T = normal((n,) * d, seed, 0)
    L = [chebyshev_vandermonde(n, n) for _ in range(d)]
    return TuckerCase(T, L, f"tucker d={d} n=m={n} chebyshev-vandermonde")


def batched_shapes(batch: int = 512, d: int = 3, lo: int = 8, hi: int = 64,
                   seed: int = SEED + 4):
    m = rng(seed, 0).integers(lo, hi + 1, size=(batch, d))
    n = np.ceil(1.5 * m).astype(np.int64)
    return m.astype(np.int64), n


def batched(batch: int = 512, d: int = 3, lo: int = 8, hi: int = 64,
            seed: int = SEED + 4) -> BatchedCase:
    m, n = batched_shapes(batch, d, lo, hi, seed)
    case = BatchedCase(m, n)
    cache = {}
    for b in range(batch):
        case.T.append(normal(tuple(int(v) for v in m[b]), seed, 1 + b))
        Ls = []
        for mu in range(d):
            key = (int(m[b, mu]), int(n[b, mu]))
            if key not in cache:
                cache[key] = barycentric_matrix(key[0], uniform_points(key[1]))
            Ls.append(cache[key])
        case.L.append(Ls)
    return case


def adjoint(n: int = 48, d: int = 4, seed: int = SEED + 5):
    T = normal((n,) * d, seed, 0)
    L = [normal((n, n), seed, 1 + k) for k in range(d)]
    target = normal((n,) * d, seed, 10)
    return TuckerCase(T, L, f"adjoint d={d} n=m={n}"), target


def tucker_flops(m, n, order=None) -> float:
    """Algorithmic flops sum_mu 2 n_mu m_mu prod(other current sizes) for the
    chain applied in ``order`` (default 0..d-1)."""
    d = len(m)
    order = list(range(d)) if order is None else list(order)
    cur = [int(v) for v in m]
    fl = 0.0
    for mu in order:
        other = 1
        for k in range(d):
            if k != mu:
                other *= cur[k]
        fl += 2.0 * n[mu] * cur[mu] * other
        cur[mu] = int(n[mu])
    return fl


def runge(points):
    """Runge function 1 / (1 + 16 sum_mu x_mu^2) on the Cartesian grid of the
    given 1-D point sets (Fortran-ordered tensor)."""
    s = None
    for mu, p in enumerate(points):
        shape = [1] * len(points)
        shape[mu] = len(p)
        term = (np.asarray(p) ** 2).reshape(shape, order="F")
        s = term if s is None else s + term
    return np.asfortranarray(1.0 / (1.0 + 16.0 * s))


def rel_err_max(x, ref) -> float:
    """Max-norm relative error ||x - ref||_inf / ||ref||_inf."""
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = float(np.max(np.abs(ref))) if ref.size else 0.0
    num = float(np.max(np.abs(x - ref))) if ref.size else 0.0
    if den == 0.0:
        return num
    return num / den



@dataclass
class SemilinearCase:
    """u_t = Laplace(u) + 1 / (1 + u^2) + Phi(t, x) on [0, 1]^3, homogeneous
    Dirichlet, u_0 = prod_mu x_mu (1 - x_mu), exact solution e^t u_0
    (Section 4.5, Eq. (semilinear))."""
    n: tuple
    tau: float
    nsteps: int
    x: list                # interior points x_j = j h, h = 1 / (n + 1)
    A: list                # dense FD Laplacians tridiag(1, -2, 1) / h^2
    M: list                # I / d - tau A_mu: M = M_d (+) ... (+) M_1
    P: list                # I - tau A_mu: ADI preconditioner P_d (x) ... (x) P_1
    U0: np.ndarray
    LU0: np.ndarray        # Laplacian of u_0 (its FD Laplacian is the same: u_0 is quadratic per axis)

    def phi(self, t: float) -> np.ndarray:
        """Phi = u_t - Laplace(u) - 1 / (1 + u^2) at u = e^t u_0."""
        et = np.exp(t)
        return np.asfortranarray(et * (self.U0 - self.LU0) - 1.0 / (1.0 + (et * self.U0) ** 2))

    def exact(self, t: float) -> np.ndarray:
        return np.asfortranarray(np.exp(t) * self.U0)


def semilinear(n=(40, 44, 48), tau: float = 0.01, tstar: float = 1.0) -> SemilinearCase:
    d = len(n)
    x = [np.arange(1, k + 1) / (k + 1.0) for k in n]
    A = [tridiag_dense(k, (k + 1.0) ** 2, -2.0 * (k + 1.0) ** 2, (k + 1.0) ** 2) for k in n]
    M = [np.asfortranarray(np.eye(k) / d - tau * a) for k, a in zip(n, A)]
    P = [np.asfortranarray(np.eye(k) - tau * a) for k, a in zip(n, A)]
    g = [xx * (1.0 - xx) for xx in x]

    def outer(vs):
        out = vs[0]
        for v in vs[1:]:
            out = np.multiply.outer(out, v)
        return np.asfortranarray(out)

    U0 = outer(g)
    LU0 = np.zeros(tuple(n), order="F")
    for mu in range(d):
        LU0 += outer([(-2.0 * np.ones(k)) if nu == mu else g[nu] for nu, k in enumerate(n)])
    nsteps = int(round(tstar / tau))
    return SemilinearCase(tuple(n), tau, nsteps, x, A, M, P, U0, np.asfortranarray(LU0))
