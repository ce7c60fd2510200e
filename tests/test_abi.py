"""Host-side checks of the C ABI: the library loads, exports every symbol
include/kron.h declares, and validates arguments without touching a GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "kron.h")


def _declared_symbols():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"KRON_API\s+[\w\s\*]*?\b(kron_\w+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "kron_build", os.path.join(ROOT, "paper_2112_11238_gb300", "build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    path = mod.build()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    syms = _declared_symbols()
    for name in ("kron_mump", "kron_tucker", "kron_tucker_adjoint", "kron_expkronsum_step",
                 "kron_batched_run", "kron_expm"):
        assert name in syms


def test_library_exports_every_declared_symbol(lib):
    missing = [s for s in _declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_covers_every_symbol(lib):
    import paper_2112_11238_gb300 as kron
    assert sorted(kron.EXPORTS) == _declared_symbols()


def _i64(v):
    return (ctypes.c_int64 * len(v))(*v)


def test_status_strings(lib):
    lib.kron_status_string.restype = ctypes.c_char_p
    assert lib.kron_status_string(0) == b"KRON_OK"
    assert lib.kron_status_string(6) == b"KRON_ERR_TIMEOUT"


def test_plan_validation_and_order(lib):
    h = ctypes.c_void_p()
    assert lib.kron_plan_create(ctypes.byref(h), 0, _i64([1]), _i64([1]), 0, 0, 0) == 1
    assert lib.kron_plan_create(ctypes.byref(h), 7, _i64([1] * 7), _i64([1] * 7), 0, 0, 0) == 1
    assert lib.kron_plan_create(ctypes.byref(h), 2, _i64([3, 0]), _i64([3, 3]), 0, 0, 0) == 1
    assert lib.kron_plan_create(ctypes.byref(h), 2, _i64([3, 3]), _i64([3, 3]), 5, 0, 0) == 1
    assert lib.kron_plan_create(ctypes.byref(h), 2, _i64([3, 3]), _i64([3, 3]), 0, 9, 0) == 1
    # cost-minimising order: shrink the big mode first
    assert lib.kron_plan_create(ctypes.byref(h), 3, _i64([50, 4, 4]), _i64([2, 40, 40]), 0, 2, 0) == 0
    order = (ctypes.c_int * 3)()
    assert lib.kron_plan_order(h, order) == 0
    assert list(order)[0] == 0
    lib.kron_plan_flops.restype = ctypes.c_double
    assert lib.kron_plan_flops(h) > 0
    ws = ctypes.c_size_t(0)
    assert lib.kron_plan_workspace_size(h, ctypes.byref(ws)) == 0 and ws.value > 0
    assert lib.kron_plan_destroy(h) == 0


def test_natural_order_flag(lib):
    h = ctypes.c_void_p()
    assert lib.kron_plan_create(ctypes.byref(h), 3, _i64([4, 4, 50]), _i64([40, 40, 2]), 1, 0, 2) == 0
    order = (ctypes.c_int * 3)()
    lib.kron_plan_order(h, order)
    assert list(order) == [0, 1, 2]
    lib.kron_plan_destroy(h)


def test_call_validation_without_gpu(lib):
    h = ctypes.c_void_p()
    assert lib.kron_plan_create(ctypes.byref(h), 2, _i64([3, 3]), _i64([3, 3]), 0, 0, 0) == 0
    L = (ctypes.c_void_p * 2)(8, 8)
    ld = _i64([3, 3])
    # null tensor
    assert lib.kron_tucker(h, None, L, ld, ctypes.c_void_p(8), None, ctypes.c_size_t(0), None) == 1
    # ld too small
    assert lib.kron_tucker(h, ctypes.c_void_p(8), L, _i64([2, 3]), ctypes.c_void_p(8), None, ctypes.c_size_t(0), None) == 1
    # misaligned tensor pointer
    assert lib.kron_tucker(h, ctypes.c_void_p(12), L, ld, ctypes.c_void_p(8), None, ctypes.c_size_t(0), None) == 3
    # workspace too small
    ws = ctypes.c_size_t(0)
    lib.kron_plan_workspace_size(h, ctypes.byref(ws))
    assert lib.kron_tucker(h, ctypes.c_void_p(8), L, ld, ctypes.c_void_p(8), ctypes.c_void_p(256), ctypes.c_size_t(0), None) == 4
    lib.kron_plan_destroy(h)
    # stepper needs a square plan
    assert lib.kron_plan_create(ctypes.byref(h), 2, _i64([3, 4]), _i64([3, 3]), 0, 0, 0) == 0
    assert lib.kron_expkronsum_workspace_size(h, ctypes.byref(ws)) == 1
    lib.kron_plan_destroy(h)
    # host-state stepper: null host or device state, misaligned device state
    # (checked before any copy is enqueued)
    assert lib.kron_plan_create(ctypes.byref(h), 2, _i64([3, 3]), _i64([3, 3]), 0, 6, 0) == 0
    A = (ctypes.c_void_p * 2)(8, 8)
    p8 = ctypes.c_void_p(8)
    args = (h, A, ld, ctypes.c_double(1e-3), 1)
    tail = (ctypes.c_void_p(256), ctypes.c_size_t(1 << 20), None)
    assert lib.kron_expkronsum_step_host(*args, None, p8, p8, *tail) == 1
    assert lib.kron_expkronsum_step_host(*args, p8, None, p8, *tail) == 1
    assert lib.kron_expkronsum_step_host(*args, p8, p8, None, *tail) == 1
    assert lib.kron_expkronsum_step_host(*args, p8, p8, ctypes.c_void_p(12), *tail) == 3
    lib.kron_plan_destroy(h)
    # the Kronecker-sum action needs a square plan, and V and S apart
    assert lib.kron_plan_create(ctypes.byref(h), 2, _i64([3, 4]), _i64([3, 3]), 0, 0, 0) == 0
    assert lib.kron_kronsumv_workspace_size(h, ctypes.byref(ws)) == 1
    lib.kron_plan_destroy(h)
    assert lib.kron_plan_create(ctypes.byref(h), 2, _i64([3, 3]), _i64([3, 3]), 0, 2, 0) == 0
    assert lib.kron_kronsumv_workspace_size(h, ctypes.byref(ws)) == 0 and ws.value > 0
    assert lib.kron_kronsumv(h, ctypes.c_void_p(8), L, ld, ctypes.c_void_p(8), None, ctypes.c_size_t(0), None) == 1
    assert lib.kron_kronsumv(h, ctypes.c_void_p(8), L, ld, ctypes.c_void_p(64), None, ctypes.c_size_t(0), None) == 1
    assert lib.kron_kronsumv(h, ctypes.c_void_p(8), L, ld, ctypes.c_void_p(64), ctypes.c_void_p(256),
                             ctypes.c_size_t(0), None) == 4
    lib.kron_plan_destroy(h)
    # expm size limits
    assert lib.kron_expm_workspace_size(0, ctypes.byref(ws)) == 1
    assert lib.kron_expm_workspace_size(2048, ctypes.byref(ws)) == 1
    assert lib.kron_expm_workspace_size(256, ctypes.byref(ws)) == 0


def test_error_word_and_timeout_hook_validation(lib):
    lib.kron_debug_dependency_timeout.argtypes = [ctypes.c_int, ctypes.c_double]
    # limits outside [0, 10 s] are refused; a valid call only sets host state
    assert lib.kron_debug_dependency_timeout(1, ctypes.c_double(-1.0)) == 1
    assert lib.kron_debug_dependency_timeout(1, ctypes.c_double(2e4)) == 1
    assert lib.kron_debug_dependency_timeout(0, ctypes.c_double(0.0)) == 0
    # the word needs somewhere to go
    assert lib.kron_get_device_error(None, None, 0) == 1


def test_tucker_batched_one_shot_validation(lib):
    ws = ctypes.c_size_t(0)
    m, n = _i64([8, 9, 10, 12, 14, 15]), _i64([12, 14, 15, 18, 21, 23])
    assert lib.kron_tucker_batched_workspace_size(2, 3, m, n, 1, 2, ctypes.byref(ws)) == 0 and ws.value > 0
    # plain precisions are not offered by the batched kernel
    assert lib.kron_tucker_batched_workspace_size(2, 3, m, n, 1, 0, ctypes.byref(ws)) == 2
    assert lib.kron_tucker_batched_workspace_size(0, 3, m, n, 1, 2, ctypes.byref(ws)) == 1
    # null pointer arrays are refused before anything is launched
    assert lib.kron_tucker_batched(2, 3, m, n, None, None, None, 1, 2, None, ctypes.c_size_t(0), None) == 1


def test_plan_launches_group_small_modes(lib):
    """Which mode products run fused (host logic): the d=6 n=m=20 chain of a
    split form with FP32 storage runs as groups {1,2,3}, {4,5}, {6}; FP64
    storage cannot start a group (the fused kernel reads FP32), FP32 groups
    on the CUDA cores (two modes or more, from a whole slab), FP64, the fixed-point forms and the
    unfused flag run one product per launch, and modes above 32 are never
    grouped."""
    def launches(m, n, dtype, prec, flags=0):
        h = ctypes.c_void_p()
        assert lib.kron_plan_create(ctypes.byref(h), len(m), _i64(m), _i64(n), dtype, prec, flags) == 0
        sz = (ctypes.c_int * len(m))()
        cnt = ctypes.c_int(0)
        assert lib.kron_plan_launches(h, sz, ctypes.byref(cnt)) == 0
        lib.kron_plan_destroy(h)
        return list(sz)[:cnt.value]
    d6 = [20] * 6
    for prec in (2, 3, 4):  # 3xTF32, BF16x3, BF16x6
        assert launches(d6, d6, 1, prec) == [3, 2, 1]
        assert launches(d6, d6, 1, prec, 0x4) == [1] * 6
        g = launches(d6, d6, 0, prec)
        assert g[0] == 1 and sum(g) == 6 and max(g) >= 2
    for prec in (0, 5, 6):  # FP64, FX32, FX32H
        assert launches(d6, d6, 1, prec) == [1] * 6
    # FP32 (CUDA cores): groups of two or three modes from a whole slab only
    assert launches(d6, d6, 1, 1) == [3, 1, 1, 1]
    assert launches([20, 20, 40], [20, 20, 40], 1, 1) == [2, 1]
    assert launches([40, 20, 20], [40, 20, 20], 1, 1) == [1, 1, 1]
    assert launches([20, 40, 20], [20, 40, 20], 1, 1) == [1, 1, 1]
    assert launches([40, 40, 40], [40, 40, 40], 1, 2) == [1, 1, 1]
    assert launches([40, 20, 20], [40, 20, 20], 1, 2, 0x2) == [1, 2]
    assert sum(launches([7, 9, 5, 11], [13, 4, 8, 3], 1, 2, 0x2)) == 4


def test_mump_workspace_query(lib):
    ws = ctypes.c_size_t(0)
    assert lib.kron_mump_workspace_size(3, _i64([5, 6, 7]), 1, 9, 1, 2, ctypes.byref(ws)) == 0
    assert ws.value >= 256
    assert lib.kron_mump_workspace_size(3, _i64([5, 6, 7]), 3, 9, 1, 2, ctypes.byref(ws)) == 1


@pytest.mark.parametrize("m", [1, 2, 9, 45, 69, 160])
def test_gauss_hermite_rule_matches_the_oracle(m):
    """kron_gauss_hermite (host code of the library: Golub--Welsch by implicit
    QL, reciprocal Christoffel weights) against numpy's hermgauss."""
    import numpy as np
    import oracle
    import paper_2112_11238_gb300 as kron
    beta = np.sqrt(2 * m + 1) / 4.0
    x, w = kron.gauss_hermite(m, beta)
    xr, wr = oracle.gauss_hermite(m, beta)
    assert np.max(np.abs(x - xr)) <= 1e-13 * max(1.0, np.max(np.abs(xr)))
    assert np.max(np.abs(w - wr) / wr) <= 1e-11


@pytest.mark.parametrize("m,alpha", [(1, 4.0), (3, 0.0), (31, 4.0), (105, 4.0), (64, -0.5)])
def test_gauss_laguerre_rule_matches_the_oracle(m, alpha):
    import numpy as np
    import oracle
    import paper_2112_11238_gb300 as kron
    beta = (4 * m + 2 * alpha + 2) / 11.0
    x, w = kron.gauss_laguerre(m, alpha, beta)
    xr, wr = oracle.gauss_laguerre(m, alpha, beta)
    assert np.max(np.abs(x - xr) / xr) <= 1e-12
    assert np.max(np.abs(w - wr) / wr) <= 1e-10


def test_spectral_argument_validation(lib):
    import numpy as np
    x = np.zeros(4)
    w = np.zeros(4)
    lib.kron_gauss_hermite.argtypes = [ctypes.c_int64, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p]
    lib.kron_gauss_laguerre.argtypes = [ctypes.c_int64, ctypes.c_double, ctypes.c_double, ctypes.c_void_p,
                                        ctypes.c_void_p]
    assert lib.kron_gauss_hermite(0, 1.0, x.ctypes.data, w.ctypes.data) == 1
    assert lib.kron_gauss_hermite(4, 0.0, x.ctypes.data, w.ctypes.data) == 1
    assert lib.kron_gauss_laguerre(4, -1.0, 1.0, x.ctypes.data, w.ctypes.data) == 1
    assert lib.kron_gauss_laguerre(4, 1.0, -2.0, x.ctypes.data, w.ctypes.data) == 1


def test_ctucker_validation_without_gpu(lib):
    """kron_ctucker rejects bad calls before any launch: fixed-point precisions,
    conj outside {0, 1}, null pointers, misalignment to a complex element, a
    short ld, a small workspace."""
    h = ctypes.c_void_p()
    ws = ctypes.c_size_t(0)
    L = (ctypes.c_void_p * 2)(16, 16)
    ld = _i64([3, 3])
    assert lib.kron_plan_create(ctypes.byref(h), 2, _i64([3, 3]), _i64([3, 3]), 0, 5, 0) == 0  # FX32
    assert lib.kron_ctucker_workspace_size(h, ctypes.byref(ws)) == 2
    assert lib.kron_ctucker(h, ctypes.c_void_p(16), L, ld, 0, ctypes.c_void_p(16), None, ctypes.c_size_t(0),
                            None) == 2
    lib.kron_plan_destroy(h)
    assert lib.kron_plan_create(ctypes.byref(h), 2, _i64([3, 3]), _i64([3, 3]), 0, 2, 1) == 0  # 3xTF32, trans
    assert lib.kron_ctucker_workspace_size(h, ctypes.byref(ws)) == 0 and ws.value > 0
    args = (L, ld)
    assert lib.kron_ctucker(h, ctypes.c_void_p(16), *args, 2, ctypes.c_void_p(16), None, ctypes.c_size_t(0),
                            None) == 1
    assert lib.kron_ctucker(h, None, *args, 1, ctypes.c_void_p(16), None, ctypes.c_size_t(0), None) == 1
    # complex double: 16-byte elements
    assert lib.kron_ctucker(h, ctypes.c_void_p(24), *args, 1, ctypes.c_void_p(16), None, ctypes.c_size_t(0),
                            None) == 3
    assert lib.kron_ctucker(h, ctypes.c_void_p(16), L, _i64([2, 3]), 1, ctypes.c_void_p(16), None,
                            ctypes.c_size_t(0), None) == 1
    assert lib.kron_ctucker(h, ctypes.c_void_p(16), *args, 1, ctypes.c_void_p(16), ctypes.c_void_p(256),
                            ctypes.c_size_t(0), None) == 4
    lib.kron_plan_destroy(h)


def test_spectral_matrix_validation_without_gpu(lib):
    lib.kron_hermite_functions.argtypes = [ctypes.c_int64, ctypes.c_double, ctypes.c_void_p, ctypes.c_int64,
                                           ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p]
    lib.kron_laguerre_functions.argtypes = [ctypes.c_int64, ctypes.c_double, ctypes.c_double, ctypes.c_void_p,
                                            ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int,
                                            ctypes.c_void_p]
    lib.kron_fourier_resample.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
                                          ctypes.c_void_p]
    p = ctypes.c_void_p(256)
    assert lib.kron_hermite_functions(0, 1.0, p, 4, p, 4, 0, None) == 1       # m < 1
    assert lib.kron_hermite_functions(3, -1.0, p, 4, p, 4, 0, None) == 1      # beta <= 0
    assert lib.kron_hermite_functions(3, 1.0, p, 4, p, 3, 0, None) == 1       # ldF < n
    assert lib.kron_hermite_functions(3, 1.0, p, 4, p, 2, 1, None) == 1       # ldF < m (trans)
    assert lib.kron_hermite_functions(3, 1.0, p, 4, p, 4, 2, None) == 1       # trans not 0 / 1
    assert lib.kron_hermite_functions(3, 1.0, None, 0, None, 1, 0, None) == 0  # no points: nothing to do
    assert lib.kron_laguerre_functions(3, -1.0, 1.0, p, 4, p, 4, 0, None) == 1  # alpha <= -1
    assert lib.kron_laguerre_functions(3, 0.5, 0.0, p, 4, p, 4, 0, None) == 1   # beta <= 0
    assert lib.kron_fourier_resample(0, 4, p, 4, None) == 1
    assert lib.kron_fourier_resample(3, 4, p, 3, None) == 1
    assert lib.kron_fourier_resample(3, 4, None, 4, None) == 1
