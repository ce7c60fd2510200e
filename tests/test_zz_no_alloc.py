"""kron_mump_noalloc: the mu-mode product for callers that cannot hand the
library any device memory (a host application whose pool owns the whole
device, or a loop that must not call cudaMalloc because it may synchronise
the device).  Its scratch is an array compiled into the library.

Checked through the C ABI against kron_mump (the workspace version), bit for
bit (both run the same kernels on the same image of op(L)), on two calls in a
row, for the P = 1 row maps of mode 0, middle and last modes, and transposed
L with a leading dimension above its row count; around the second call no
device memory is allocated.  This file is collected last."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2112_11238_gb300 as kron
    return torch, kron


def _i64(v):
    return (ctypes.c_int64 * len(v))(*[int(x) for x in v])


# (shape, mu, n, transL, extra leading-dimension rows)
CASES = [((37, 41, 9), 1, 50, 0, 0), ((64, 30, 33), 2, 77, 0, 0), ((45, 12, 7), 0, 60, 0, 3),
         ((20, 33, 5), 1, 29, 1, 5), ((130, 6), 0, 17, 1, 0)]


@pytest.mark.parametrize("prec,dtype", [("3xtf32", "f32"), ("bf16x6", "f64"), ("bf16x3", "f32")])
def test_noalloc_matches_workspace_mump_twice(env, prec, dtype):
    torch, kron = env
    lib = kron._lib
    tdt = torch.float32 if dtype == "f32" else torch.float64
    dcode = kron.F32 if dtype == "f32" else kron.F64
    pc = kron.PREC[prec]
    g = np.random.default_rng(5)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call, (shape, mu, n, trans, pad) in enumerate(CASES):
        d = len(shape)
        T = kron.colmajor(torch.from_numpy(np.asfortranarray(g.standard_normal(shape))).to(tdt).cuda())
        # op(L) is n x m_mu; stored as L (n x m_mu) or L^T (m_mu x n), with ld rows
        rows, cols = (shape[mu], n) if trans else (n, shape[mu])
        ld = rows + pad
        Lfull = torch.from_numpy(np.asfortranarray(g.standard_normal((ld, cols)))).to(tdt).cuda()
        Lfull = kron.colmajor(Lfull)
        out_shape = list(shape)
        out_shape[mu] = n
        S_ref = kron.empty_colmajor(out_shape, tdt, T.device)
        S_na = kron.empty_colmajor(out_shape, tdt, T.device)
        need = ctypes.c_size_t(0)
        assert lib.kron_mump_workspace_size(d, _i64(shape), mu, n, dcode, pc, ctypes.byref(need)) == 0
        ws = torch.empty(max(need.value, 256), dtype=torch.uint8, device=T.device)
        assert lib.kron_mump(d, _i64(shape), mu, n, T.data_ptr(), Lfull.data_ptr(), ld, trans, S_ref.data_ptr(),
                             dcode, pc, ws.data_ptr(), ws.numel(), stream) == 0
        # two calls in a row: the second finds the first call's scratch contents
        for rep in range(2):
            S_na.fill_(float("nan"))
            torch.cuda.synchronize()
            free0, alloc0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated()
            assert lib.kron_mump_noalloc(d, _i64(shape), mu, n, T.data_ptr(), Lfull.data_ptr(), ld, trans,
                                         S_na.data_ptr(), dcode, pc, stream) == 0
            torch.cuda.synchronize()
            if rep == 1:
                # nothing allocated by the call (the kernels are loaded by then)
                assert torch.cuda.mem_get_info()[0] == free0
                assert torch.cuda.memory_allocated() == alloc0
            assert torch.equal(S_na, S_ref), (prec, call, rep)


def test_noalloc_rejects_oversized_and_unsupported(env):
    torch, kron = env
    lib = kron._lib
    stream = ctypes.c_void_p(0)
    dummy = ctypes.c_void_p(256)
    # an image of op(L) larger than the 1 MiB scratch
    assert lib.kron_mump_noalloc(2, _i64([4, 4096]), 1, 4096, dummy, dummy, 4096, 0, dummy, kron.F32,
                                 kron.PREC["3xtf32"], stream) == 4
    # plain precisions have no split image: not offered
    assert lib.kron_mump_noalloc(2, _i64([4, 4]), 1, 4, dummy, dummy, 4, 0, dummy, kron.F64,
                                 kron.PREC["fp64"], stream) == 2
