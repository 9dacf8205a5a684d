"""gb300-rsvd: tall-skinny SVD / PCA on one GB300 (sm_103a), after arXiv:1906.12085.

Thin ctypes binding over the C ABI of ``include/rsvd.h``.  The functions keep
the C names and argument order; tensors are passed as device pointers
(``tensor.data_ptr()``) and the CUDA stream defaults to torch's current
stream.  PyTorch is used only to own device memory and streams: every step
of every solve runs in the kernels of ``libgb300rsvd.so``.  If the library
has not been built, importing the binding's functions raises; there is no
fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

__all__ = [
    "RSVD_F64", "RSVD_F32", "RSVD_BF16", "RSVD_FP8_E4M3",
    "RSVD_OK", "RSVD_ERR_ARG", "RSVD_ERR_OOM", "RSVD_ERR_CHOL", "RSVD_ERR_NOCONV", "RSVD_ERR_TIMEOUT",
    "RSVD_ERR_CUDA", "RSVD_ERR_UNSUPPORTED", "RSVD_WARN_K_GT_k", "RSVD_WARN_RANK_DEFICIENT", "RSVD_EXACT_GRAM", "RSVD_EXACT_QR_JACOBI",
    "RSVD_FLAG_NO_CENTER", "RSVD_FLAG_GKL_TWO_PASS", "RSVD_FLAG_SMALL_F32", "RSVD_FLAG_SMALL_FP64", "RsvdError", "lib", "library_path", "header_functions", "RSVD_ERR_REDUCE", "ALLREDUCE_FN",
    "allreduce_callback", "rsvd_sharded",
    "rsvd_plan_create", "rsvd_plan_destroy", "rsvd_plan_workspace_bytes", "rsvd_plan_set_flags",
    "rsvd_plan_sync", "rsvd", "svd_exact", "svd_truncated_krylov", "pca_threshold", "rsvd_plan_fro2",
    "rsvd_status_string", "check", "rsvd_plan_profile", "rsvd_plan_profile_read", "rsvd_launch_count",
    "STAGES", "svd_exact_gram_static", "RSVD_BATCH_MAX", "Completion", "rsvd_workspace_query",
    "rsvd_plan_create_in", "Batch", "rsvd_batch_create", "rsvd_batch_run", "rsvd_batch_sync",
    "rsvd_batch_destroy", "Server", "rsvd_server_create", "rsvd_server_submit", "rsvd_server_poll",
    "rsvd_server_pending", "rsvd_server_destroy", "rsvd_autotune", "rsvd_tune_lookup", "rsvd_tune_clear",
    "rsvd_quantize", "rsvd_server_submit_ex", "rsvd_plan_create_block_krylov", "rsvd_block_krylov",
    "rsvd_set_jacobi_sweep_cap",
]

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
HEADER = os.path.join(ROOT, "include", "rsvd.h")

RSVD_F64, RSVD_F32, RSVD_BF16, RSVD_FP8_E4M3 = 0, 1, 2, 3
RSVD_OK, RSVD_ERR_ARG, RSVD_ERR_OOM, RSVD_ERR_CHOL, RSVD_ERR_NOCONV = 0, -1, -2, -3, -4
RSVD_ERR_TIMEOUT, RSVD_ERR_CUDA, RSVD_ERR_UNSUPPORTED, RSVD_WARN_K_GT_k = -5, -6, -8, 1
RSVD_WARN_RANK_DEFICIENT = 2
RSVD_ERR_REDUCE = -9
RSVD_EXACT_GRAM, RSVD_EXACT_QR_JACOBI = 0, 1
RSVD_FLAG_NO_CENTER = 1
RSVD_FLAG_GKL_TWO_PASS = 2
RSVD_FLAG_SMALL_F32 = 4
RSVD_FLAG_SMALL_FP64 = 8
RSVD_BATCH_MAX = 256
# tracing stages (RSVD_STAGE_* in include/rsvd.h)
STAGES = ("center", "ax", "atx", "orth", "small", "finish")


class Completion(ctypes.Structure):
    """rsvd_completion of include/rsvd.h."""
    _fields_ = [("id", ctypes.c_int64), ("status", ctypes.c_int), ("K", ctypes.c_int), ("batch", ctypes.c_int),
                ("submit_ms", ctypes.c_double), ("start_ms", ctypes.c_double), ("done_ms", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class RsvdError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        super().__init__(f"{what}: status {status} ({rsvd_status_string(status)})")
        self.status = status


def library_path() -> str:
    return os.path.join(HERE, "libgb300rsvd.so")


_lib = None


def lib() -> ctypes.CDLL:
    """Load libgb300rsvd.so; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_1906_12085_gb300.build.build()")
    L = ctypes.CDLL(path)
    i64, i32, vp, dp = ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)
    L.rsvd_plan_create.argtypes = [ctypes.POINTER(vp), i64, i64, i32, i32, i32, i32, vp]
    L.rsvd_plan_destroy.argtypes = [vp]
    L.rsvd_plan_workspace_bytes.argtypes = [vp]
    L.rsvd_plan_workspace_bytes.restype = ctypes.c_size_t
    L.rsvd_plan_set_flags.argtypes = [vp, ctypes.c_uint]
    L.rsvd_plan_sync.argtypes = [vp]
    L.rsvd.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    L.svd_exact.argtypes = [vp, vp, i32, vp, vp, vp]
    L.svd_truncated_krylov.argtypes = [vp, vp, vp, i32, vp, vp, vp]
    L.pca_threshold.argtypes = [vp, ctypes.c_double, ctypes.POINTER(i32)]
    L.rsvd_plan_fro2.argtypes = [vp, dp]
    L.rsvd_plan_profile.argtypes = [vp, i32]
    L.rsvd_plan_profile_read.argtypes = [vp, dp, ctypes.POINTER(i32), i32]
    L.rsvd_launch_count.argtypes = []
    L.rsvd_launch_count.restype = ctypes.c_uint64
    L.svd_exact_gram_static.argtypes = [vp, i64, i64, i32, vp, vp, vp, vp]
    L.svd_exact_gram_static.restype = i32
    L.rsvd_status_string.argtypes = [i32]
    L.rsvd_status_string.restype = ctypes.c_char_p
    sz = ctypes.c_size_t
    L.rsvd_workspace_query.argtypes = [i64, i64, i32, i32, i32, i32, ctypes.POINTER(sz)]
    L.rsvd_plan_create_in.argtypes = [ctypes.POINTER(vp), i64, i64, i32, i32, i32, i32, vp, vp, sz]
    L.rsvd_batch_create.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(vp), vp]
    L.rsvd_batch_run.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp),
                                 ctypes.POINTER(vp), ctypes.POINTER(vp)]
    L.rsvd_batch_sync.argtypes = [vp, ctypes.POINTER(i32)]
    L.rsvd_batch_destroy.argtypes = [vp]
    L.rsvd_server_create.argtypes = [ctypes.POINTER(vp), sz, i32, i32]
    L.rsvd_server_submit.argtypes = [vp, i64, i64, i64, i32, i32, i32, ctypes.c_double, vp, vp, vp, vp, vp]
    L.rsvd_server_poll.argtypes = [vp, ctypes.POINTER(Completion), i32]
    L.rsvd_server_submit_ex.argtypes = [vp, i64, i64, i64, i32, i32, i32, i32, ctypes.c_double, vp, vp, vp, vp, vp, vp]
    L.rsvd_server_pending.argtypes = [vp]
    L.rsvd_server_destroy.argtypes = [vp]
    L.rsvd_autotune.argtypes = [vp, vp, vp, i32, ctypes.POINTER(i32), ctypes.POINTER(i32)]
    L.rsvd_tune_lookup.argtypes = [i64, i64, i32, i32, ctypes.POINTER(i32), ctypes.POINTER(i32)]
    L.rsvd_quantize.argtypes = [vp, i64, i64, i64, i32, vp, vp, vp]
    L.rsvd_tune_clear.argtypes = []
    L.rsvd_plan_create_block_krylov.argtypes = [ctypes.POINTER(vp), i64, i64, i32, i32, i32, i32, vp]
    L.rsvd_block_krylov.argtypes = [vp, vp, vp, vp, vp, vp]
    L.rsvd_tune_clear.restype = None
    L.rsvd_set_jacobi_sweep_cap.argtypes = [i32]
    L.rsvd_sharded.argtypes = [vp, i64, vp, vp, vp, vp, vp, ALLREDUCE_FN, vp]
    for f in ("rsvd_plan_create", "rsvd_plan_destroy", "rsvd_plan_set_flags", "rsvd_plan_sync", "rsvd",
              "svd_exact", "svd_truncated_krylov", "pca_threshold", "rsvd_plan_fro2", "rsvd_plan_profile",
              "rsvd_plan_profile_read", "rsvd_workspace_query", "rsvd_plan_create_in", "rsvd_batch_create",
              "rsvd_batch_run", "rsvd_batch_sync", "rsvd_batch_destroy", "rsvd_server_create",
              "rsvd_server_submit", "rsvd_server_poll", "rsvd_server_pending", "rsvd_server_destroy",
              "rsvd_autotune", "rsvd_tune_lookup", "rsvd_quantize", "rsvd_server_submit_ex",
              "rsvd_plan_create_block_krylov", "rsvd_block_krylov", "rsvd_set_jacobi_sweep_cap",
              "rsvd_sharded"):
        getattr(L, f).restype = i32
    _lib = L
    return L


def header_functions() -> list[str]:
    """Names of the functions include/rsvd.h declares."""
    with open(HEADER) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b([a-z_][a-z0-9_]*)\s*\(", text)) -
                  {"if", "while", "for", "sizeof", "return", "defined", "int"})


def rsvd_set_jacobi_sweep_cap(cap: int) -> int:
    """Process-wide Jacobi sweep cap (0 restores the defaults)."""
    return lib().rsvd_set_jacobi_sweep_cap(int(cap))


def rsvd_status_string(status: int) -> str:
    try:
        return lib().rsvd_status_string(int(status)).decode()
    except Exception:  # message formatting must not mask the original error
        return "?"


def check(status: int, what: str = "call", allow=(RSVD_OK,)) -> int:
    if status not in allow:
        raise RsvdError(status, what)
    return status


def _ptr(t) -> int | None:
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if not t.is_contiguous():
        raise ValueError("tensors must be contiguous (row-major)")
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Plan:
    """Owning handle of an rsvd_plan_t (destroyed on close / garbage collection)."""

    def __init__(self, handle: int, m, n, k, p, q, dtype):
        self.handle = handle
        self.m, self.n, self.k, self.p, self.q, self.dtype = m, n, k, p, q, dtype

    @property
    def l(self):
        return self.k + self.p

    def close(self):
        if self.handle:
            lib().rsvd_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class BlockKrylovPlan(Plan):
    """Plan of the block Krylov method: blocks of b columns, iters + 1 of them (W = (iters + 1) b)."""

    def __init__(self, handle: int, m, n, k, b, iters, dtype):
        super().__init__(handle, m, n, k, 0, iters, dtype)
        self.b, self.iters = b, iters

    @property
    def l(self):
        return self.b

    @property
    def W(self):
        return (self.iters + 1) * self.b


def rsvd_plan_create(m: int, n: int, k: int, p: int, q: int, dtype: int = RSVD_F32, stream=None) -> Plan:
    h = ctypes.c_void_p()
    st = lib().rsvd_plan_create(ctypes.byref(h), m, n, k, p, q, dtype, _stream(stream))
    check(st, "rsvd_plan_create")
    return Plan(h.value, m, n, k, p, q, dtype)


def rsvd_plan_destroy(plan: Plan) -> int:
    plan.close()
    return RSVD_OK


def rsvd_plan_workspace_bytes(plan: Plan) -> int:
    return int(lib().rsvd_plan_workspace_bytes(plan.handle))


def rsvd_plan_set_flags(plan: Plan, flags: int) -> int:
    return lib().rsvd_plan_set_flags(plan.handle, flags)


def rsvd_plan_sync(plan: Plan) -> int:
    return lib().rsvd_plan_sync(plan.handle)


def rsvd(plan: Plan, A, col_scales, Omega, S, U, V) -> int:
    return lib().rsvd(plan.handle, _ptr(A), _ptr(col_scales), _ptr(Omega), _ptr(S), _ptr(U), _ptr(V))


# int allreduce(double *values, int64_t count, void *ctx): values <- their sum over all ranks
ALLREDUCE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.c_int64, ctypes.c_void_p)


def allreduce_callback(reduce_inplace):
    """Wrap reduce_inplace(buf) -- buf a float64 numpy array that must be replaced by its
    elementwise sum over all ranks -- as the library's rsvd_allreduce_fn (returns 1 on an
    exception).  Keep the returned object alive while the library may call it."""
    def cb(values, count, ctx):
        try:
            reduce_inplace(np.ctypeslib.as_array(values, shape=(int(count),)))
            return 0
        except Exception:
            return 1
    return ALLREDUCE_FN(cb)


def rsvd_sharded(plan: Plan, m_total: int, A, Omega, S, U, V, reduce_inplace) -> int:
    """Row-sharded rsvd of this rank's rows A (see include/rsvd.h); reduce_inplace as for
    allreduce_callback (e.g. shard.dist_allreduce() over a torch.distributed group)."""
    fn = allreduce_callback(reduce_inplace)
    return lib().rsvd_sharded(plan.handle, int(m_total), _ptr(A), _ptr(Omega), _ptr(S), _ptr(U), _ptr(V), fn, None)


def rsvd_plan_create_block_krylov(m: int, n: int, k: int, b: int, iters: int, dtype: int = RSVD_F32,
                                  stream=None) -> Plan:
    """Plan of the block Krylov method: blocks of b columns, iters + 1 of them."""
    h = ctypes.c_void_p()
    st = lib().rsvd_plan_create_block_krylov(ctypes.byref(h), m, n, k, b, iters, dtype, _stream(stream))
    check(st, "rsvd_plan_create_block_krylov")
    return BlockKrylovPlan(h.value, m, n, k, b, iters, dtype)


def rsvd_block_krylov(plan: Plan, A, Omega, S, U, V) -> int:
    return lib().rsvd_block_krylov(plan.handle, _ptr(A), _ptr(Omega), _ptr(S), _ptr(U), _ptr(V))


def svd_exact(plan: Plan, A, method: int, S, U, V) -> int:
    return lib().svd_exact(plan.handle, _ptr(A), int(method), _ptr(S), _ptr(U), _ptr(V))


def svd_truncated_krylov(plan: Plan, A, v1, steps: int, S, U, V) -> int:
    return lib().svd_truncated_krylov(plan.handle, _ptr(A), _ptr(v1), int(steps), _ptr(S), _ptr(U), _ptr(V))


def pca_threshold(plan: Plan, t: float) -> tuple[int, int]:
    K = ctypes.c_int(0)
    st = lib().pca_threshold(plan.handle, float(t), ctypes.byref(K))
    return st, int(K.value)


def rsvd_plan_fro2(plan: Plan) -> float:
    f = ctypes.c_double(0.0)
    check(lib().rsvd_plan_fro2(plan.handle, ctypes.byref(f)), "rsvd_plan_fro2")
    return f.value


def rsvd_plan_profile(plan: Plan, enable: bool) -> int:
    return lib().rsvd_plan_profile(plan.handle, 1 if enable else 0)


def rsvd_plan_profile_read(plan: Plan) -> dict:
    """Per-stage {name: (milliseconds, groups)} since the previous read (synchronises)."""
    n = len(STAGES)
    ms = (ctypes.c_double * n)()
    cnt = (ctypes.c_int * n)()
    check(lib().rsvd_plan_profile_read(plan.handle, ms, cnt, n), "rsvd_plan_profile_read")
    return {STAGES[i]: (ms[i], cnt[i]) for i in range(n)}


def rsvd_launch_count() -> int:
    return int(lib().rsvd_launch_count())


def svd_exact_gram_static(A, dtype: int, S, U, V, stream=None) -> int:
    """Gram-route exact SVD with no device allocation (scratch in the library's static array).

    For callers that cannot allocate device memory; see include/rsvd.h.
    Synchronises the stream before returning."""
    m, n = A.shape
    return lib().svd_exact_gram_static(_ptr(A), m, n, int(dtype), _ptr(S), _ptr(U), _ptr(V), _stream(stream))


# ------------------------------------------------------------- batching and serving
def rsvd_workspace_query(m: int, n: int, k: int, p: int, q: int, dtype: int = RSVD_F32) -> tuple[int, int]:
    """(status, bytes of device workspace a plan of these sizes needs)."""
    b = ctypes.c_size_t(0)
    st = lib().rsvd_workspace_query(m, n, k, p, q, dtype, ctypes.byref(b))
    return st, int(b.value)


class _PlanIn(Plan):
    """A plan on caller-owned workspace; keeps the workspace tensor alive."""

    def __init__(self, handle, m, n, k, p, q, dtype, workspace):
        super().__init__(handle, m, n, k, p, q, dtype)
        self.workspace = workspace


def rsvd_plan_create_in(m: int, n: int, k: int, p: int, q: int, dtype: int, stream, workspace) -> Plan:
    """rsvd_plan_create on `workspace` (a device tensor of at least rsvd_workspace_query bytes)."""
    h = ctypes.c_void_p()
    nbytes = workspace.numel() * workspace.element_size()
    st = lib().rsvd_plan_create_in(ctypes.byref(h), m, n, k, p, q, dtype, _stream(stream), _ptr(workspace), nbytes)
    check(st, "rsvd_plan_create_in")
    return _PlanIn(h.value, m, n, k, p, q, dtype, workspace)


def _ptrs(ts):
    arr = (ctypes.c_void_p * len(ts))()
    for i, t in enumerate(ts):
        arr[i] = _ptr(t)
    return arr


class Batch:
    """Owning handle of an rsvd_batch_t; keeps its plans alive."""

    def __init__(self, handle, plans):
        self.handle = handle
        self.plans = list(plans)

    def close(self):
        if self.handle:
            lib().rsvd_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def rsvd_batch_create(plans, stream=None) -> Batch:
    h = ctypes.c_void_p()
    arr = (ctypes.c_void_p * len(plans))(*[p.handle for p in plans])
    check(lib().rsvd_batch_create(ctypes.byref(h), len(plans), arr, _stream(stream)), "rsvd_batch_create")
    return Batch(h.value, plans)


def rsvd_batch_run(batch: Batch, A, Omega, S, U, V) -> int:
    return lib().rsvd_batch_run(batch.handle, _ptrs(A), _ptrs(Omega), _ptrs(S), _ptrs(U), _ptrs(V))


def rsvd_batch_sync(batch: Batch) -> tuple[int, list[int]]:
    sts = (ctypes.c_int * len(batch.plans))()
    st = lib().rsvd_batch_sync(batch.handle, sts)
    return st, list(sts)


def rsvd_batch_destroy(batch: Batch) -> int:
    batch.close()
    return RSVD_OK


class Server:
    """Owning handle of an rsvd_server_t."""

    def __init__(self, handle):
        self.handle = handle

    def close(self):
        if self.handle:
            lib().rsvd_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def rsvd_server_create(hbm_bytes: int, max_batch: int = 16, max_inflight: int = 8) -> Server:
    h = ctypes.c_void_p()
    check(lib().rsvd_server_create(ctypes.byref(h), int(hbm_bytes), max_batch, max_inflight), "rsvd_server_create")
    return Server(h.value)


def rsvd_server_submit(server: Server, rid: int, k: int, p: int, q: int, t: float, A, Omega, S, U, V) -> int:
    m, n = A.shape
    return lib().rsvd_server_submit(server.handle, int(rid), m, n, k, p, q, float(t), _ptr(A), _ptr(Omega), _ptr(S),
                                    _ptr(U), _ptr(V))


def rsvd_server_submit_ex(server: Server, rid: int, k: int, p: int, q: int, dtype: int, t: float, A, col_scales,
                          Omega, S, U, V) -> int:
    m, n = A.shape
    return lib().rsvd_server_submit_ex(server.handle, int(rid), m, n, k, p, q, int(dtype), float(t), _ptr(A),
                                       _ptr(col_scales), _ptr(Omega), _ptr(S), _ptr(U), _ptr(V))


def rsvd_server_poll(server: Server, max_out: int = 256) -> list[dict]:
    """Progress the server; the completions it returns (dicts of rsvd_completion fields)."""
    buf = (Completion * max_out)()
    w = lib().rsvd_server_poll(server.handle, buf, max_out)
    if w < 0:
        raise RsvdError(w, "rsvd_server_poll")
    return [buf[i].as_dict() for i in range(w)]


def rsvd_server_pending(server: Server) -> int:
    return int(lib().rsvd_server_pending(server.handle))


def rsvd_server_destroy(server: Server) -> int:
    server.close()
    return RSVD_OK


def rsvd_autotune(plan: Plan, A, Omega, concurrency: int = 1) -> tuple[int, int, int]:
    """(status, nn_ctas, tn_ctas): tune the products' decomposition for the plan's bucket."""
    a, b = ctypes.c_int(0), ctypes.c_int(0)
    st = lib().rsvd_autotune(plan.handle, _ptr(A), _ptr(Omega), concurrency, ctypes.byref(a), ctypes.byref(b))
    return st, a.value, b.value


def rsvd_tune_lookup(m: int, n: int, k: int, p: int) -> tuple[int, int, int]:
    a, b = ctypes.c_int(0), ctypes.c_int(0)
    st = lib().rsvd_tune_lookup(m, n, k, p, ctypes.byref(a), ctypes.byref(b))
    return st, a.value, b.value


def rsvd_tune_clear() -> None:
    lib().rsvd_tune_clear()


def rsvd_quantize(A, dtype: int, Aq, col_scales=None, stream=None) -> int:
    """Store the float32 matrix A (device) as bfloat16 or e4m3 codes in Aq (see include/rsvd.h)."""
    m, n = A.shape
    return lib().rsvd_quantize(_ptr(A), m, n, n, int(dtype), _ptr(Aq), _ptr(col_scales), _stream(stream))
