"""C-ABI checks that need no GPU: the library loads, exports every function
include/rsvd.h declares, and rejects invalid arguments before touching CUDA."""
import ctypes
import subprocess

import pytest

import paper_1906_12085_gb300 as g


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1906_12085_gb300 import build
    build.build()


def test_library_exports_every_header_function():
    names = g.header_functions()
    assert {"rsvd_plan_create", "rsvd", "svd_exact", "svd_truncated_krylov", "pca_threshold"} <= set(names)
    L = g.lib()
    missing = [f for f in names if not hasattr(L, f)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", g.library_path()], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    assert set(names) <= exported


def test_binding_covers_every_header_function():
    """The Python layer keeps the C names: one callable per declared function, and every
    library symbol has its argument types declared (no implicit int conversions)."""
    names = g.header_functions()
    assert [n for n in names if not callable(getattr(g, n, None))] == []
    L = g.lib()
    assert [n for n in names if getattr(getattr(L, n), "argtypes", None) is None] == []
    assert set(names) <= set(g.__all__)


def test_library_has_no_oracle_dependency():
    """The product library links neither the oracle library nor any of its symbols."""
    out = subprocess.run(["nm", "-D", g.library_path()], capture_output=True, text=True).stdout
    assert "orc_" not in out
    ldd = subprocess.run(["ldd", g.library_path()], capture_output=True, text=True).stdout
    assert "liboracle" not in ldd


@pytest.mark.parametrize("args", [
    (10, 20, 1, 0, 0, g.RSVD_F32),      # m < n
    (100, 20, 0, 0, 0, g.RSVD_F32),     # k < 1
    (100, 20, 15, 10, 0, g.RSVD_F32),   # l = k + p > n
    (100, 20, 5, -1, 0, g.RSVD_F32),    # p < 0
    (100, 20, 5, 1, -2, g.RSVD_F32),    # q < 0
    (0, 0, 1, 0, 0, g.RSVD_F32),
])
def test_plan_create_rejects_bad_sizes(args):
    h = ctypes.c_void_p(12345)
    st = g.lib().rsvd_plan_create(ctypes.byref(h), *args, None)
    assert st == g.RSVD_ERR_ARG
    assert h.value is None


def test_plan_create_rejects_unbuilt_dtypes():
    h = ctypes.c_void_p()
    for dt in (g.RSVD_FP8_E4M3, 7):
        assert g.lib().rsvd_plan_create(ctypes.byref(h), 100, 20, 4, 2, 1, dt, None) == g.RSVD_ERR_UNSUPPORTED
    # bfloat16 plans need rows of whole 16-byte units (n a multiple of 8) and l <= 288
    assert g.lib().rsvd_plan_create(ctypes.byref(h), 100, 20, 4, 2, 1, g.RSVD_BF16, None) == g.RSVD_ERR_UNSUPPORTED
    assert g.lib().rsvd_plan_create(ctypes.byref(h), 1000, 512, 280, 16, 1, g.RSVD_BF16, None) == \
        g.RSVD_ERR_UNSUPPORTED
    # float32 randomized solves up to l = 288, float64 up to 112
    assert g.lib().rsvd_plan_create(ctypes.byref(h), 1000, 512, 280, 16, 1, g.RSVD_F32, None) == \
        g.RSVD_ERR_UNSUPPORTED
    assert g.lib().rsvd_plan_create(ctypes.byref(h), 1000, 512, 100, 16, 1, g.RSVD_F64, None) == \
        g.RSVD_ERR_UNSUPPORTED


@pytest.mark.parametrize("args,want", [
    ((10, 20, 1, 4, 0, g.RSVD_F32), g.RSVD_ERR_ARG),        # m < n
    ((100, 20, 0, 4, 1, g.RSVD_F32), g.RSVD_ERR_ARG),       # k < 1
    ((100, 20, 4, 0, 1, g.RSVD_F32), g.RSVD_ERR_ARG),       # b < 1
    ((100, 20, 4, 4, -1, g.RSVD_F32), g.RSVD_ERR_ARG),      # iters < 0
    ((100, 20, 13, 4, 2, g.RSVD_F32), g.RSVD_ERR_ARG),      # k > W = (iters + 1) b
    ((100, 20, 4, 8, 2, g.RSVD_F32), g.RSVD_ERR_ARG),       # W > n
    ((1000, 512, 8, 120, 0, g.RSVD_F32), g.RSVD_ERR_UNSUPPORTED),   # block Gram beyond one CTA (b > 112)
    ((1000, 512, 100, 100, 2, g.RSVD_F32), g.RSVD_ERR_UNSUPPORTED),  # W = 300 > 288
    ((1000, 512, 8, 60, 1, g.RSVD_F64), g.RSVD_ERR_UNSUPPORTED),    # float64: W = 120 > 112
    ((1000, 512, 8, 16, 1, g.RSVD_BF16), g.RSVD_ERR_UNSUPPORTED),   # float32 / float64 only
])
def test_block_krylov_plan_rejects_bad_sizes(args, want):
    h = ctypes.c_void_p(12345)
    assert g.lib().rsvd_plan_create_block_krylov(ctypes.byref(h), *args, None) == want
    assert h.value is None
    assert g.lib().rsvd_block_krylov(None, None, None, None, None, None) == g.RSVD_ERR_ARG


def test_null_plan_arguments():
    L = g.lib()
    assert L.rsvd_plan_destroy(None) == g.RSVD_OK
    assert L.rsvd_plan_workspace_bytes(None) == 0
    assert L.rsvd(None, None, None, None, None, None, None) == g.RSVD_ERR_ARG
    assert L.svd_exact(None, None, 0, None, None, None) == g.RSVD_ERR_ARG
    assert L.svd_truncated_krylov(None, None, None, 1, None, None, None) == g.RSVD_ERR_ARG
    K = ctypes.c_int(0)
    assert L.pca_threshold(None, 0.9, ctypes.byref(K)) == g.RSVD_ERR_ARG
    assert L.rsvd_plan_sync(None) == g.RSVD_ERR_ARG
    assert g.rsvd_status_string(g.RSVD_ERR_CHOL) == "Cholesky breakdown"


def test_workspace_query_and_create_in_argument_errors():
    L = g.lib()
    st, b = g.rsvd_workspace_query(10, 20, 1, 0, 0)          # m < n
    assert st == g.RSVD_ERR_ARG and b == 0
    st, b = g.rsvd_workspace_query(100, 20, 4, 2, 1, g.RSVD_FP8_E4M3)
    assert st == g.RSVD_ERR_UNSUPPORTED
    st, b = g.rsvd_workspace_query(1000, 64, 8, 4, 1)
    assert st == g.RSVD_OK and b > 0 and b % 256 == 0
    h = ctypes.c_void_p()
    assert L.rsvd_plan_create_in(ctypes.byref(h), 1000, 64, 8, 4, 1, g.RSVD_F32, None, None, b) == g.RSVD_ERR_ARG
    assert L.rsvd_plan_create_in(ctypes.byref(h), 1000, 64, 8, 4, 1, g.RSVD_F32, None, 4096 + 16, b) == g.RSVD_ERR_ARG
    assert L.rsvd_plan_create_in(None, 1000, 64, 8, 4, 1, g.RSVD_F32, None, 4096, b) == g.RSVD_ERR_ARG
    assert h.value is None


def test_batch_and_server_argument_errors():
    L = g.lib()
    h = ctypes.c_void_p()
    assert L.rsvd_batch_create(ctypes.byref(h), 0, None, None) == g.RSVD_ERR_ARG
    assert L.rsvd_batch_create(ctypes.byref(h), g.RSVD_BATCH_MAX + 1, None, None) == g.RSVD_ERR_ARG
    assert L.rsvd_batch_run(None, None, None, None, None, None) == g.RSVD_ERR_ARG
    assert L.rsvd_batch_sync(None, None) == g.RSVD_ERR_ARG
    assert L.rsvd_batch_destroy(None) == g.RSVD_OK
    assert L.rsvd_server_create(ctypes.byref(h), 0, 4, 2) == g.RSVD_ERR_ARG
    assert L.rsvd_server_create(ctypes.byref(h), 1 << 20, 0, 2) == g.RSVD_ERR_ARG
    assert L.rsvd_server_create(ctypes.byref(h), 1 << 20, 4, 0) == g.RSVD_ERR_ARG
    assert L.rsvd_server_submit(None, 0, 100, 10, 2, 1, 1, 0.9, None, None, None, None, None) == g.RSVD_ERR_ARG
    assert L.rsvd_server_poll(None, None, 0) == g.RSVD_ERR_ARG
    assert L.rsvd_server_pending(None) == 0
    assert L.rsvd_server_destroy(None) == g.RSVD_OK


def test_autotune_argument_errors():
    L = g.lib()
    a, b = ctypes.c_int(7), ctypes.c_int(7)
    assert L.rsvd_autotune(None, None, None, 1, ctypes.byref(a), ctypes.byref(b)) == g.RSVD_ERR_ARG
    g.rsvd_tune_clear()
    assert g.rsvd_tune_lookup(1000, 64, 8, 8)[0] == g.RSVD_ERR_ARG
    assert g.rsvd_tune_lookup(0, 64, 8, 8)[0] == g.RSVD_ERR_ARG


def test_sharded_flags_and_sweep_cap_argument_errors():
    """Entry points of the sharded solve, the plan flags and the sweep cap reject bad
    arguments before any CUDA call."""
    L = g.lib()
    fn = g.allreduce_callback(lambda buf: None)
    assert L.rsvd_sharded(None, 100, None, None, None, None, None, fn, None) == g.RSVD_ERR_ARG
    assert L.rsvd_plan_set_flags(None, g.RSVD_FLAG_NO_CENTER) == g.RSVD_ERR_ARG
    assert g.rsvd_set_jacobi_sweep_cap(-1) == g.RSVD_ERR_ARG
    assert g.rsvd_set_jacobi_sweep_cap(0) == g.RSVD_OK          # restores the defaults
    assert g.rsvd_status_string(g.RSVD_ERR_REDUCE) == "the reduction over ranks failed"
    assert g.rsvd_status_string(g.RSVD_WARN_RANK_DEFICIENT).startswith("numerically rank-deficient")
    # distinct flag bits, all accepted by the library's mask
    flags = [g.RSVD_FLAG_NO_CENTER, g.RSVD_FLAG_GKL_TWO_PASS, g.RSVD_FLAG_SMALL_F32, g.RSVD_FLAG_SMALL_FP64]
    assert len(set(flags)) == 4 and all(f & (f - 1) == 0 for f in flags)


def test_allreduce_callback_marshalling():
    """The reduction callback sees the library's buffer as a float64 array it can change in
    place, and reports an exception as a non-zero return."""
    seen = []

    def double_it(buf):
        seen.append(buf.dtype)
        buf *= 2.0

    fn = g.allreduce_callback(double_it)
    arr = (ctypes.c_double * 5)(1, 2, 3, 4, 5)
    assert fn(ctypes.cast(arr, ctypes.POINTER(ctypes.c_double)), 5, None) == 0
    assert list(arr) == [2, 4, 6, 8, 10] and str(seen[0]) == "float64"

    def boom(buf):
        raise RuntimeError("peer gone")
    bad = g.allreduce_callback(boom)
    assert bad(ctypes.cast(arr, ctypes.POINTER(ctypes.c_double)), 5, None) == 1
