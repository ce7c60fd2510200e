"""GPU parity of the HLF transform matrices (normalized scaled Hermite and
generalized Laguerre functions, Fourier resampling) against the oracle, their
orthonormality at large m, and the paper's HLF experiment run through the
library (transform matrices and both Tucker operators on the GPU)."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kron():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2112_11238_gb300 as k
    return k


def host(t):
    return np.asfortranarray(t.detach().cpu().numpy())


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("trans", [False, True])
@pytest.mark.parametrize("m,beta,n", [(1, 1.0, 7), (9, 1.3, 41), (69, 2.1, 301), (150, 3.1, 257)])
def test_hermite_functions_match_the_oracle(kron, m, beta, n, trans):
    x = np.linspace(-4.0, 4.0, n)
    F = host(kron.hermite_functions(m, beta, x, trans=trans))
    ref = oracle.hermite_functions(m, beta, x)
    assert _rel(F, ref.T if trans else ref) <= 1e-12


@pytest.mark.parametrize("trans", [False, True])
@pytest.mark.parametrize("m,alpha,beta,n", [(1, 4.0, 1.0, 5), (8, 0.0, 0.7, 33), (105, 4.0, 39.2, 301),
                                           (40, 1.5, 3.0, 100)])
def test_laguerre_functions_match_the_oracle(kron, m, alpha, beta, n, trans):
    x = np.linspace(0.0, 11.0, n)
    F = host(kron.laguerre_functions(m, alpha, beta, x, trans=trans))
    ref = oracle.laguerre_functions(m, alpha, beta, x)
    assert _rel(F, ref.T if trans else ref) <= 1e-12


@pytest.mark.parametrize("m,n", [(1, 4), (8, 301), (38, 301), (7, 20), (64, 64)])
def test_fourier_resample_matches_the_oracle(kron, m, n):
    assert _rel(host(kron.fourier_resample(m, n)), oracle.fourier_resample(m, n)) <= 1e-13


@pytest.mark.parametrize("kind", ["hermite", "laguerre"])
def test_transform_matrices_are_orthonormal_at_large_m(kron, kind):
    """m = 400: the plain recurrence would underflow far out; the library's
    scaled one keeps Psi diag(w) Psi^T = I."""
    import torch
    m = 400
    if kind == "hermite":
        beta = np.sqrt(2 * m + 1) / 4.0
        x, w = kron.gauss_hermite(m, beta)
        Psi = kron.hermite_functions(m, beta, x, trans=True)
    else:
        alpha, beta = 4.0, (4 * m + 10) / 11.0
        x, w = kron.gauss_laguerre(m, alpha, beta)
        Psi = kron.laguerre_functions(m, alpha, beta, x, trans=True)
    P = Psi.cpu().numpy()
    G = P @ np.diag(w) @ P.T
    assert np.max(np.abs(G - np.eye(m))) <= 1e-10
    assert torch.isfinite(Psi).all()


def _golden_hlf():
    import os
    rows = []
    with open(os.path.join(os.path.dirname(__file__), "golden", "fig_spectral_hlf_accuracy.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                m1, m2, m3, acc = line.split()
                rows.append(((int(m1), int(m2), int(m3)), float(acc)))
    return rows


@pytest.mark.parametrize("prec", ["fp64", "3xtf32"])
def test_hlf_decomposition_on_the_gpu_reproduces_the_paper(kron, prec):
    """The HLF experiment with the library's quadrature, transform matrices and
    Tucker operators: FW x_1 Psi_1 x_2 Psi_2, then x_1 Phi_1 x_2 Phi_2 x_3 Phi_3
    on 301^3 points, against f; the accuracies of the paper's figure."""
    import torch
    alpha, b1, b2, a3, b3, n = 4.0, 4.0, 11.0, -1.0, 1.0, 301
    dev = torch.device("cuda")
    x1 = -b1 + 2 * b1 * np.arange(n) / n
    x2 = b2 * np.arange(n) / n
    x3 = a3 + (b3 - a3) * np.arange(n) / n
    F = oracle.hlf_function(x1[:, None, None], x2[None, :, None], x3[None, None, :])
    for (m1, m2, m3), acc in _golden_hlf():
        beta1 = np.sqrt(2 * m1 + 1) / b1
        beta2 = (4 * m2 + 2 * alpha + 2) / b2
        xi1, w1 = kron.gauss_hermite(m1, beta1)
        xi2, w2 = kron.gauss_laguerre(m2, alpha, beta2)
        xi3 = a3 + (b3 - a3) * np.arange(m3) / m3
        FW = oracle.hlf_function(xi1[:, None, None], xi2[None, :, None], xi3[None, None, :]) \
            * w1[:, None, None] * w2[None, :, None]
        FWd = kron.colmajor(torch.from_numpy(np.asfortranarray(FW)).to(dev))
        Psi = [kron.hermite_functions(m1, beta1, xi1, trans=True),
               kron.laguerre_functions(m2, alpha, beta2, xi2, trans=True),
               kron.colmajor(torch.eye(m3, dtype=torch.float64, device=dev))]
        Fhat = kron.tucker(FWd, Psi, prec=prec)
        Phi = [kron.hermite_functions(m1, beta1, x1), kron.laguerre_functions(m2, alpha, beta2, x2),
               kron.fourier_resample(m3, n)]
        Ft = host(kron.tucker(Fhat, Phi, prec=prec))
        err = float(np.max(np.abs(Ft - F)) / np.max(np.abs(F)))
        # the split form adds its own rounding (budget 2e-6 relative) to the truncation error
        slack = 2e-3 * acc + (0.0 if prec == "fp64" else 2e-6)
        assert abs(err - acc) <= slack, (prec, (m1, m2, m3), err, acc)
    assert kron.device_error() == 0
