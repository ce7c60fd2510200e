"""GPU parity of the complex Tucker operator (Eq. (tuckerop) over C, op(L) = L,
L^T, L^*, conj(L); the conjugate transposes are the paper's cttucker) against
the complex128 oracle: ragged shapes with P = 1 and P > 1 modes (one- and
two-level index maps), every precision of the path, complex128 and complex64
storage; the DFT property at a larger size."""
import numpy as np
import pytest

import oracle
from gpu_util import TOL, rel_err, tol

pytestmark = pytest.mark.gpu

RNG = np.random.default_rng(4242)
PRECS = ["fp64", "fp32", "3xtf32", "bf16x3", "bf16x6"]
OPS = [(False, False), (True, False), (True, True), (False, True)]


def crnd(*s):
    return np.asfortranarray(RNG.standard_normal(s) + 1j * RNG.standard_normal(s))


@pytest.fixture(scope="module")
def kron():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2112_11238_gb300 as k
    return k


def to_dev_c(a, dtype=None):
    import torch
    import paper_2112_11238_gb300 as k
    t = torch.from_numpy(np.asfortranarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return k.colmajor(t.cuda())


def to_host_c(t):
    return np.asfortranarray(t.detach().cpu().numpy().astype(np.complex128))


SHAPES = [((7,), (5,)), ((37, 19), (40, 19)), ((9, 33, 17), (9, 20, 30)), ((130, 5, 3), (7, 5, 3)),
          ((4, 6, 5, 3), (5, 6, 4, 7))]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("trans,conj", OPS)
@pytest.mark.parametrize("m,n", SHAPES)
def test_ctucker_matches_oracle(kron, m, n, trans, conj, prec):
    T = crnd(*m)
    Ls = [crnd(m[k], n[k]) if trans else crnd(n[k], m[k]) for k in range(len(m))]
    ref = oracle.ctucker(T, Ls, transL=trans, conj=conj)
    S = kron.ctucker(to_dev_c(T), [to_dev_c(L) for L in Ls], prec=prec, trans=trans, conj=conj)
    err = rel_err(to_host_c(S), ref)
    # each complex product sums 2 m_mu real products
    assert err <= tol(prec, 2 * max(m)), (prec, m, n, trans, conj, err)
    assert kron.device_error() == 0


@pytest.mark.parametrize("prec", ["fp32", "3xtf32", "bf16x6"])
def test_ctucker_complex64_storage(kron, prec):
    import torch
    m, n = (11, 23, 6), (13, 9, 6)
    T = crnd(*m)
    Ls = [crnd(m[k], n[k]) for k in range(3)]
    T64 = to_dev_c(T, torch.complex64)
    L64 = [to_dev_c(L, torch.complex64) for L in Ls]
    ref = oracle.ctucker(to_host_c(T64), [to_host_c(L) for L in L64], transL=True, conj=True)
    S = kron.cttucker(T64, L64, prec=prec)
    assert S.dtype == torch.complex64
    assert rel_err(to_host_c(S), ref) <= max(TOL[prec], 1e-6)


@pytest.mark.parametrize("prec", ["fp64", "3xtf32", "bf16x6"])
def test_cttucker_dft_at_96_cubed(kron, prec):
    """Psi_mu = the 96-point DFT matrix: cttucker gives 96^3 times the inverse
    FFT of T (numpy.fft.ifftn) at a size the oracle's loops would not reach."""
    T = crnd(96, 96, 96)
    F = np.exp(-2j * np.pi * np.outer(np.arange(96), np.arange(96)) / 96)
    ref = np.fft.ifftn(T) * T.size
    S = kron.cttucker(to_dev_c(T), [to_dev_c(F)] * 3, prec=prec)
    assert rel_err(to_host_c(S), ref) <= (1e-12 if prec == "fp64" else 2e-6), prec


@pytest.mark.parametrize("prec", ["fx32", "fx32h"])
def test_ctucker_fixed_point_is_unsupported(kron, prec):
    T = crnd(4, 5)
    Ls = [crnd(3, 4), crnd(2, 5)]
    with pytest.raises(kron.KronError) as e:
        kron.ctucker(to_dev_c(T), [to_dev_c(L) for L in Ls], prec=prec)
    assert e.value.code == 2  # KRON_ERR_UNSUPPORTED
