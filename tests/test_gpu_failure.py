"""Failure detection on the GPU without faulting it: a bounded wait is made to
run out, and the kernel reports it through the device error word.

The persistent tensor-core kernel waits, inside one launch, for the tiles of
the jobs a job reads (the modes of the batched Tucker operators).  The test
hook makes every such wait ask for one tile more than its job has, so it can
end only at its time limit (here 20 ms); the kernel then latches the timeout
bit, carries on and returns, and the context stays usable.  The data waited
for was complete, so the results are still the operator's."""
import ctypes

import numpy as np
import pytest

import oracle
from gpu_util import TOL, rel_err, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kron():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2112_11238_gb300 as k
    return k


def test_dependency_wait_timeout_is_reported_and_cleared(kron):
    import torch
    g = np.random.default_rng(11)
    batch, d = 5, 3
    m = g.integers(8, 40, size=(batch, d))
    n = np.ceil(1.5 * m).astype(np.int64)
    T = [np.asfortranarray(g.standard_normal(tuple(m[b]))) for b in range(batch)]
    L = [[np.asfortranarray(g.standard_normal((n[b, k], m[b, k]))) for k in range(d)] for b in range(batch)]
    dev = torch.device("cuda")
    Ts = [to_dev(t, torch.float32) for t in T]
    Ls = [[to_dev(x, torch.float32) for x in row] for row in L]
    Ss = [kron.empty_colmajor(tuple(int(v) for v in n[b]), torch.float32, dev) for b in range(batch)]
    plan = kron.BatchedPlan(m, n, torch.float32, "3xtf32")
    ws = plan.workspace(dev)
    plan.bind(Ts, Ls, Ss, ws)
    assert kron.device_error() == 0

    plan.run(ws)
    first = [s.clone() for s in Ss]
    assert kron.device_error() == 0

    kron.debug_dependency_timeout(True, 20.0)
    try:
        for s in Ss:
            s.fill_(float("nan"))
        plan.run(ws)
        torch.cuda.synchronize()
    finally:
        kron.debug_dependency_timeout(False)
    # the status through the C ABI, then the word itself; reading clears it
    code = ctypes.c_int(0)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert kron._lib.kron_get_device_error(stream, ctypes.byref(code), 0) == 6  # KRON_ERR_TIMEOUT
    assert code.value & 1
    assert kron.device_error() & 1
    assert kron.device_error() == 0
    # the tiles went ahead after the wait: same results as before
    for a, b in zip(first, Ss):
        assert torch.equal(a, b)

    # normal operation again, and still the operator's values
    for s in Ss:
        s.fill_(float("nan"))
    plan.run(ws)
    assert kron.device_error() == 0
    for b in range(batch):
        assert torch.equal(first[b], Ss[b])
        assert rel_err(to_host(Ss[b]), oracle.tucker(T[b], L[b])) <= TOL["3xtf32"]
