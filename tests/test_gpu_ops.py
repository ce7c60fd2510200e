"""GPU parity of the mu-mode product, the Tucker operator and expm against the
FP64 oracle, on small and ragged shapes (several tiles, ragged tails, P = 1
and Q = 1 slabs, n != m, transposed L), every precision, both storage types."""
import numpy as np
import pytest

import oracle
from gpu_util import TOL, rel_err, to_dev, to_host, tol

pytestmark = pytest.mark.gpu

RNG = np.random.default_rng(2024)
PRECS = ["fp64", "fp32", "3xtf32", "bf16x3", "bf16x6", "fx32", "fx32h"]


def rnd(*s):
    return np.asfortranarray(RNG.standard_normal(s))


@pytest.fixture(scope="module")
def kron():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2112_11238_gb300 as k
    return k


MUMP_CASES = [
    ((7,), 0, 5), ((37, 3), 0, 19), ((3, 37), 1, 40), ((130, 5, 3), 0, 7),
    ((9, 33, 17), 1, 33), ((5, 6, 300), 2, 12), ((129, 2, 2), 1, 257), ((20, 20, 20, 3), 2, 20),
    ((1, 1, 5), 2, 1), ((64, 64), 1, 64), ((17, 70), 0, 33),
    # several N-tiles whose width is not a power of two
    ((14, 54, 8), 0, 81), ((14, 54, 8), 1, 65), ((30, 33, 20), 2, 129), ((9, 40, 7), 1, 200),
]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("shape,mu,n", MUMP_CASES)
def test_mump_matches_oracle(kron, shape, mu, n, prec):
    import torch
    T = rnd(*shape)
    L = rnd(n, shape[mu])
    ref = oracle.mump(T, L, mu)
    S = kron.mump(to_dev(T), to_dev(L), mu, prec=prec)
    err = rel_err(to_host(S), ref)
    assert err <= tol(prec, shape[mu]), (prec, shape, mu, n, err)
    assert kron.device_error() == 0


@pytest.mark.parametrize("prec", ["fp64", "3xtf32", "bf16x6"])
def test_mump_transposed(kron, prec):
    T = rnd(11, 23, 5)
    L = rnd(23, 30)  # op(L) = L^T is 30 x 23
    ref = oracle.mump(T, L, 1, transL=True)
    S = kron.mump(to_dev(T), to_dev(L), 1, trans=True, prec=prec)
    assert rel_err(to_host(S), ref) <= TOL[prec]


@pytest.mark.parametrize("prec", ["3xtf32", "bf16x6", "fp32"])
def test_mump_float32_storage(kron, prec):
    import torch
    T = rnd(40, 33, 9)
    L = rnd(17, 33)
    ref = oracle.mump(T, L, 1)
    S = kron.mump(to_dev(T, torch.float32), to_dev(L, torch.float32), 1, prec=prec)
    assert S.dtype == torch.float32
    assert rel_err(to_host(S), ref) <= max(TOL[prec], 1e-6)


TUCKER_CASES = [
    ((5, 7), (9, 3)), ((13, 4, 9), (6, 11, 2)), ((33, 31, 29), (35, 30, 28)),
    ((6, 5, 4, 3), (3, 4, 5, 6)), ((4, 3, 5, 2, 3), (2, 5, 3, 4, 2)), ((4,) * 6, (5,) * 6),
    ((100, 1, 7), (1, 50, 7)),
]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("m,n", TUCKER_CASES)
def test_tucker_matches_oracle(kron, m, n, prec):
    T = rnd(*m)
    Ls = [rnd(n[k], m[k]) for k in range(len(m))]
    ref = oracle.tucker(T, Ls)
    S = kron.tucker(to_dev(T), [to_dev(L) for L in Ls], prec=prec)
    assert tuple(S.shape) == tuple(n)
    err = rel_err(to_host(S), ref)
    assert err <= tol(prec, sum(m)), (prec, m, n, err)


# chains whose small modes run as fused groups (up to three neighbouring
# modes with m, n <= 32 per launch, intermediates on chip): groups at the
# start (contiguous slabs) and after larger modes (p-blocks with a ragged
# tail), single small modes, n != m, sizes of 1
FUSED_CASES = [
    ((20, 20, 20), (20, 20, 20)), ((7, 9, 5, 11), (13, 4, 8, 3)), ((32, 1, 17), (5, 32, 2)),
    ((40, 12, 13, 14), (40, 9, 30, 7)), ((3, 50, 6, 7, 8), (4, 50, 9, 2, 31)), ((5,) * 6, (6, 4, 7, 3, 5, 2)),
    ((33, 31, 3), (29, 30, 31)), ((1, 1, 1), (32, 1, 16)), ((16, 16, 16, 16, 16), (16,) * 5),
    ((1, 6, 7), (9, 5, 4)), ((3, 1, 9, 2), (5, 7, 1, 6)),
]


@pytest.mark.parametrize("prec", ["3xtf32", "bf16x3", "bf16x6"])
@pytest.mark.parametrize("m,n", FUSED_CASES)
def test_fused_groups_match_oracle_and_unfused(kron, m, n, prec):
    import torch
    T = rnd(*m)
    Ls = [rnd(n[k], m[k]) for k in range(len(m))]
    ref = oracle.tucker(T, Ls)
    Tf = to_dev(T, torch.float32)
    Lf = [to_dev(L, torch.float32) for L in Ls]
    S = kron.tucker(Tf, Lf, prec=prec, natural_order=True)
    U = kron.tucker(Tf, Lf, prec=prec, natural_order=True, fused=False)
    ref32 = oracle.tucker(to_host(Tf), [to_host(L) for L in Lf])
    assert rel_err(to_host(S), ref32) <= TOL[prec], (prec, m, n, rel_err(to_host(S), ref32))
    assert rel_err(to_host(U), ref32) <= TOL[prec]
    assert rel_err(to_host(S), ref) <= max(TOL[prec], 1e-6)
    assert kron.device_error() == 0


@pytest.mark.parametrize("io", ["f32", "f64"])
@pytest.mark.parametrize("trans", [False, True])
@pytest.mark.parametrize("m,n", FUSED_CASES)
def test_fused_fp32_groups_match_oracle_and_unfused_bitwise(kron, m, n, trans, io):
    """FP32 groups on the CUDA cores: every output is the same ascending chain
    of fused multiply-adds as in the per-mode kernel, over the same FP32
    intermediates, so the fused and unfused chains agree bit for bit."""
    import torch
    dt = torch.float32 if io == "f32" else torch.float64
    T = rnd(*m)
    Ls = [rnd(m[k], n[k]) if trans else rnd(n[k], m[k]) for k in range(len(m))]
    Td = to_dev(T, dt)
    Ld = [to_dev(L, dt) for L in Ls]
    S = kron.tucker(Td, Ld, prec="fp32", trans=trans, natural_order=True)
    U = kron.tucker(Td, Ld, prec="fp32", trans=trans, natural_order=True, fused=False)
    assert torch.equal(S, U), (m, n, trans, io)
    ref = oracle.tucker(to_host(Td), [(to_host(L).T.copy(order="F") if trans else to_host(L)) for L in Ld])
    assert rel_err(to_host(S), ref) <= tol("fp32", sum(m)), (m, n, rel_err(to_host(S), ref))
    assert kron.device_error() == 0


KSV_SHAPES = [(7,), (37, 19), (9, 33, 17), (130, 5, 3), (20, 20, 20, 3), (3, 4, 5, 6, 7)]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("shape", KSV_SHAPES)
def test_kronsumv_matches_oracle(kron, shape, prec):
    """sum_mu V x_mu L_mu against the oracle (Eq. (actkron))."""
    V = rnd(*shape)
    Ls = [rnd(n, n) for n in shape]
    ref = oracle.kronsumv(V, Ls)
    S = kron.kronsumv(to_dev(V), [to_dev(L) for L in Ls], prec=prec)
    err = rel_err(to_host(S), ref)
    assert err <= tol(prec, max(shape)), (prec, shape, err)
    assert kron.device_error() == 0


@pytest.mark.parametrize("prec", ["fp64", "3xtf32", "fx32", "fx32h"])
def test_kronsumv_transposed_and_float32(kron, prec):
    import torch
    shape = (11, 23, 5)
    V = rnd(*shape)
    Ls = [rnd(n, n) for n in shape]
    ref_t = oracle.kronsumv(V, [L.T.copy(order="F") for L in Ls])
    S = kron.kronsumv(to_dev(V), [to_dev(L) for L in Ls], prec=prec, trans=True)
    assert rel_err(to_host(S), ref_t) <= TOL[prec]
    if prec != "fp64":
        S32 = kron.kronsumv(to_dev(V).float(), [to_dev(L).float() for L in Ls], prec=prec)
        ref32 = oracle.kronsumv(to_host(to_dev(V).float()), [to_host(to_dev(L).float()) for L in Ls])
        assert S32.dtype == torch.float32
        assert rel_err(to_host(S32), ref32) <= max(TOL[prec], 1e-6)


def _wc(n):
    """A well-conditioned n x n matrix (I plus a small random part)."""
    return np.asfortranarray(np.eye(n) + 0.3 * RNG.standard_normal((n, n)) / np.sqrt(n))


IT_SHAPES = [(7,), (37, 19), (9, 33, 17), (130, 5, 3), (20, 20, 20, 3)]


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("shape", IT_SHAPES)
def test_itucker_matches_oracle(kron, shape, prec):
    """V x_mu P_mu^{-1} (FP64 inverses on the GPU, chain in prec) against the
    oracle's mode-by-mode LU solves (Eq. (preconnd))."""
    V = rnd(*shape)
    Ps = [_wc(n) for n in shape]
    ref = oracle.itucker(V, Ps)
    S = kron.itucker(to_dev(V), [to_dev(P) for P in Ps], prec=prec)
    err = rel_err(to_host(S), ref)
    assert err <= 2 * tol(prec, max(shape)), (prec, shape, err)
    assert kron.device_error() == 0


@pytest.mark.parametrize("prec", ["fp32", "3xtf32", "bf16x3", "bf16x6", "fx32", "fx32h"])
def test_itucker_refinement_reaches_fp64_accuracy(kron, prec):
    """FP64-residual iterative refinement of the low-precision chain."""
    shape = (9, 33, 17)
    V = rnd(*shape)
    Ps = [_wc(n) for n in shape]
    ref = oracle.itucker(V, Ps)
    e0 = rel_err(to_host(kron.itucker(to_dev(V), [to_dev(P) for P in Ps], prec=prec)), ref)
    e3 = rel_err(to_host(kron.itucker(to_dev(V), [to_dev(P) for P in Ps], prec=prec, refine=3)), ref)
    assert e3 <= 1e-12 and e3 < e0 / 100, (prec, e0, e3)


@pytest.mark.parametrize("prec", ["fp64", "3xtf32", "fx32", "fx32h"])
def test_itucker_transposed_and_float32(kron, prec):
    import torch
    shape = (11, 23, 5)
    V = rnd(*shape)
    Ps = [_wc(n) for n in shape]
    ref_t = oracle.itucker(V, Ps, transL=True)
    S = kron.itucker(to_dev(V), [to_dev(P) for P in Ps], prec=prec, trans=True, refine=1)
    assert rel_err(to_host(S), ref_t) <= 1e-12
    V32, P32 = to_dev(V).float(), [to_dev(P).float() for P in Ps]
    ref32 = oracle.itucker(to_host(V32), [to_host(P) for P in P32])
    S32 = kron.itucker(V32, P32, prec=prec, refine=2)
    assert S32.dtype == torch.float32
    assert rel_err(to_host(S32), ref32) <= 2e-7  # FP32 storage of S


def test_itucker_singular_matrix_sets_the_numeric_flag(kron):
    shape = (6, 5)
    V = rnd(*shape)
    Ps = [np.zeros((6, 6), order="F"), _wc(5)]
    kron.itucker(to_dev(V), [to_dev(P) for P in Ps], prec="fp64")
    assert kron.device_error() & 2
    assert kron.device_error() == 0  # cleared by the read


@pytest.mark.parametrize("prec", ["fx32", "fx32h"])
def test_fx32_rows_far_below_the_largest_row_sum(kron, prec):
    """Rows of op(L_mu) whose magnitude is far below the largest row sum: in
    the fixed-point chain their products are scaled down (a negative shift)
    before rounding, and must keep their own scale (Eq. (tuckerop))."""
    T = rnd(9, 10, 11)
    Ls = [rnd(8, 9), rnd(7, 10), rnd(6, 11)]
    for L in Ls:  # whichever mode runs last, the others produce fixed point
        L[3, :] *= 2.0 ** -20
        L[5, :] *= 2.0 ** -12
    ref = oracle.tucker(T, Ls)
    S = kron.tucker(to_dev(T), [to_dev(L) for L in Ls], prec=prec)
    assert rel_err(to_host(S), ref) <= TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "3xtf32"])
def test_tucker_transposed_plan(kron, prec):
    m, n = (7, 9, 5), (4, 10, 6)
    T = rnd(*m)
    Ls = [rnd(m[k], n[k]) for k in range(3)]   # op(L) = L^T
    ref = oracle.tucker(T, Ls, transL=True)
    S = kron.tucker(to_dev(T), [to_dev(L) for L in Ls], prec=prec, trans=True)
    assert rel_err(to_host(S), ref) <= TOL[prec]


def test_identity_returns_input_exactly_fp64(kron):
    T = rnd(9, 8, 7)
    S = kron.tucker(to_dev(T), [to_dev(np.eye(k)) for k in T.shape], prec="fp64")
    np.testing.assert_array_equal(to_host(S), T)


@pytest.mark.parametrize("n", [1, 5, 64, 256])
def test_expm_matches_closed_form(kron, n):
    import workloads as W
    sub, diag, sup = W.fd_advection_diffusion(n)
    tau = 1e-4
    A = W.tridiag_dense(n, sub, diag, sup)
    ref = oracle.expm_tridiag_toeplitz(n, sub, diag, sup, tau)
    E = kron.expm(to_dev(A), tau)
    assert rel_err(to_host(E), ref) <= 1e-12
    assert kron.device_error() == 0


def test_expm_random_matrix(kron):
    A = rnd(12, 12)
    ref = oracle.expm_taylor(A, 0.37)
    E = kron.expm(to_dev(A), 0.37)
    assert rel_err(to_host(E), ref) <= 1e-12


@pytest.mark.parametrize("prec", ["fx32h", "3xtf32", "fp64"])
def test_stepper_host_state_matches_device_state(kron, prec):
    """kron_expkronsum_step_host (state copied in beside the exponentials,
    copied back after the steps) gives the device-state stepper's bits, in
    place and into a separate host buffer, and the oracle's values."""
    import torch
    import workloads as W
    c = W.stepper(n=24, tau=1e-4, nsteps=3)
    dev = torch.device("cuda")
    A = [to_dev(a) for a in c.A]
    plan = kron.StepperPlan([c.n] * 3, torch.float64, prec)
    ws = plan.workspace(dev)
    U_ref = plan.step(to_dev(c.U0), A, c.tau, c.nsteps, ws=ws)
    torch.cuda.synchronize()
    U_in = kron.pinned_colmajor(c.U0.shape)
    U_in.copy_(torch.from_numpy(c.U0))
    U_out = kron.pinned_colmajor(c.U0.shape)
    plan.step_host(U_in, A, c.tau, c.nsteps, U_out=U_out, ws=ws)
    torch.cuda.synchronize()
    assert torch.equal(U_out, U_ref.cpu())
    np.testing.assert_array_equal(U_in.numpy(), c.U0)  # the input is left as it was
    plan.step_host(U_in, A, c.tau, c.nsteps, ws=ws)  # in place
    torch.cuda.synchronize()
    assert torch.equal(U_in, U_ref.cpu())
    E = oracle.expm_tridiag_toeplitz(c.n, *c.tri, c.tau)
    ref = oracle.expkronsum_steps(c.U0, [E] * 3, c.nsteps)
    assert rel_err(U_out.numpy(), ref) <= tol(prec, 3 * c.n)
    assert kron.device_error() == 0
