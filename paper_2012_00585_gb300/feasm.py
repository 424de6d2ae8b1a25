"""ctypes binding of libfeasm (include/feasm.h), same names as the C ABI.

Argument marshalling only: every step of the assembly runs in the CUDA
library.  Device buffers are passed as torch CUDA tensors (or raw integer
device addresses); streams as torch.cuda.Stream, raw cudaStream_t integers,
or None for torch's current stream.  There is no CPU fallback: if the CUDA
library cannot be loaded, every call raises.
"""

import ctypes
import os
import threading

from . import _build

FE_OK = 0
FE_ERR_INVALID_ARG = -1
FE_ERR_DOF_RANGE = -2
FE_ERR_DUP_DOF = -3
FE_ERR_OVERFLOW = -4
FE_ERR_OOM = -5
FE_ERR_ADMISSION = -6
FE_ERR_TIMEOUT = -7
FE_ERR_DEVICE = -8
FE_ERR_NOT_BUILT = -9
FE_ERR_UNSUPPORTED = -10
FE_ERR_NOT_FOUND = -11
FE_ERR_CANCELLED = -12
FE_MAX_NLOC = 128

FE_PATTERN_CSR = 0x1
FE_PATTERN_CRAC = 0x2
FE_PATTERN_MAP_CSR = 0x4
FE_PATTERN_MAP_CRAC = 0x8
FE_PATTERN_ADJ = 0x10
FE_PATTERN_ALL = 0x1F

FE_ATOMIC = 0
FE_DETERMINISTIC = 1
FE_COLOURED = 2
FE_ROWLOCK = 3

FE_KNOB_GATHER_KERNEL = 0
FE_KNOB_GATHER_BATCH = 1
FE_KNOB_GATHER_WARPS = 2
FE_KNOB_ATOMIC_KERNEL = 3
FE_KNOB_ATOMIC_WARPS = 4
FE_KNOB_ATOMIC_ORDER = 5
FE_KNOB_LOCK_SPIN = 6
FE_KNOB_SPMV_LANES = 7
FE_KNOB_COUNT = 8

FE_FORMAT_CSR = 0
FE_FORMAT_CRAC = 1
FE_SCHED_WARP_PER_ELEMENT = 1
FE_SCHED_THREAD_PER_ENTRY = 2
FE_SCHED_BLOCK_PER_ELEMENT = 3
FE_SCHED_WARP_PER_ROW = 4
FE_SCHED_WARP_PER_ELEMENT_TMA = 5

_lib = None
_lock = threading.Lock()


class FeError(RuntimeError):
    def __init__(self, code, where=""):
        self.code = int(code)
        msg = fe_strerror(code) if _lib is not None else f"error {code}"
        detail = ""
        if self.code == FE_ERR_DEVICE and _lib is not None:
            detail = " [" + _lib.fe_last_cuda_error().decode() + "]"
        super().__init__(f"{where}: {msg} ({code}){detail}")


class fe_pattern_info(ctypes.Structure):
    _fields_ = [
        ("n_elem", ctypes.c_int64),
        ("n_loc", ctypes.c_int32),
        ("map_bytes", ctypes.c_int32),
        ("n_dofs", ctypes.c_int64),
        ("nnz", ctypes.c_int64),
        ("n_ca", ctypes.c_int64),
        ("n_elem_runs", ctypes.c_int64),
        ("max_row_len", ctypes.c_int32),
        ("max_degree", ctypes.c_int32),
        ("flags", ctypes.c_uint32),
        ("block", ctypes.c_int32),
        ("uniform_runs", ctypes.c_int32),
        ("atomic_order", ctypes.c_int32),
        ("device_bytes", ctypes.c_int64),
    ]


class fe_schedule(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("tile", ctypes.c_int32)]


class fe_batch_item(ctypes.Structure):
    _fields_ = [("pattern", ctypes.c_void_p), ("elem_mats", ctypes.c_void_p), ("values", ctypes.c_void_p),
                ("times_ns", ctypes.c_void_p)]


FE_STATE_PENDING = 0
FE_STATE_ADMITTED = 1
FE_STATE_RUNNING = 2
FE_STATE_DONE = 3
FE_STATE_FAILED = 4
FE_STATE_CANCELLED = 5


class fe_request(ctypes.Structure):
    _fields_ = [("pattern_key", ctypes.c_uint64), ("n_elem", ctypes.c_int64), ("dofs_per_elem", ctypes.c_int32),
                ("format", ctypes.c_int32), ("n_dofs", ctypes.c_int64), ("elem_dofs", ctypes.c_void_p),
                ("elem_mats", ctypes.c_void_p), ("k_ref", ctypes.c_void_p), ("seed", ctypes.c_uint64),
                ("mode", ctypes.c_int32), ("reserved", ctypes.c_int32), ("ready_event", ctypes.c_void_p),
                ("deadline_s", ctypes.c_double)]


class fe_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("state", ctypes.c_int32), ("cold", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("nnz", ctypes.c_int64), ("row_ptr", ctypes.c_void_p),
                ("col_idx", ctypes.c_void_p), ("values", ctypes.c_void_p), ("t_submit_us", ctypes.c_double),
                ("t_admit_us", ctypes.c_double), ("t_start_us", ctypes.c_double), ("t_done_us", ctypes.c_double),
                ("t_ready_us", ctypes.c_double)]


class fe_server_stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("submitted", "admitted", "completed", "failed", "cancelled",
                                              "launches", "batched_requests", "patterns_built", "evictions",
                                              "bytes_in_use", "budget_bytes", "cached_patterns", "rebuilds",
                                              "expired", "admission_waits", "peak_bytes_in_use")] + \
        [("alloc_ms_total", ctypes.c_double), ("alloc_ms_max", ctypes.c_double)] + \
        [(n, ctypes.c_int64) for n in ("n_pending", "n_to_build", "n_ready", "n_big_jobs", "n_running",
                                       "n_inflight_groups")]


class fe_span(ctypes.Structure):
    _fields_ = [("start_ms", ctypes.c_double), ("end_ms", ctypes.c_double), ("stream", ctypes.c_int32),
                ("n_requests", ctypes.c_int32)]


def library_path() -> str:
    return _build.LIB_DEBUG if os.environ.get("FEASM_DEBUG") == "1" else _build.LIB


def load():
    """Load the CUDA library (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        # FEASM_DEBUG=1: the build with every device index check compiled in
        path = _build.build(debug=os.environ.get("FEASM_DEBUG") == "1")
        if not os.path.exists(path):
            raise RuntimeError(f"libfeasm not found at {path}; the CUDA path has no fallback")
        lib = ctypes.CDLL(path)
        vp, i64, i32, u32, i = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint32, ctypes.c_int
        pp = ctypes.POINTER(vp)
        sig = {
            "fe_create": (i, [pp, i, ctypes.c_size_t]),
            "fe_create_ex": (i, [pp, i, ctypes.c_size_t, ctypes.c_size_t]),
            "fe_destroy": (i, [vp]),
            "fe_strerror": (ctypes.c_char_p, [i]),
            "fe_last_cuda_error": (ctypes.c_char_p, []),
            "fe_kernel_launches": (ctypes.c_uint64, []),
            "fe_debug_checks": (i, []),
            "fe_device_status": (i, [vp, vp]),
            "fe_tune_set": (i, [vp, i, i]),
            "fe_tune_get": (i, [vp, i, ctypes.POINTER(i)]),
            "fe_pattern_build": (i, [vp, i64, i32, i64, vp, u32, vp, pp]),
            "fe_pattern_free": (i, [vp]),
            "fe_pattern_free_async": (i, [vp, vp]),
            "fe_pattern_csr_noalloc": (i, [i64, i32, i64, vp, vp, vp, i64, ctypes.POINTER(i64), vp]),
            "fe_pattern_csr": (i, [vp, pp, pp, ctypes.POINTER(i64)]),
            "fe_pattern_crac": (i, [vp, pp, pp, ctypes.POINTER(i64)]),
            "fe_pattern_adjacency": (i, [vp, ctypes.POINTER(i32), pp, pp]),
            "fe_pattern_info_get": (i, [vp, ctypes.POINTER(fe_pattern_info)]),
            "fe_pattern_colour": (i, [vp, vp, vp, ctypes.POINTER(i32)]),
            "fe_pattern_colours": (i, [vp, ctypes.POINTER(i32), pp]),
            "fe_assemble_csr": (i, [vp, vp, vp, vp, i, i, vp]),
            "fe_assemble_crac": (i, [vp, vp, vp, vp, i, i, vp]),
            "fe_spmv_csr": (i, [vp, vp, vp, vp, vp, vp]),
            "fe_spmv_crac": (i, [vp, vp, vp, vp, vp, vp]),
            "fe_assemble_batch": (i, [vp, ctypes.POINTER(fe_batch_item), i32, i32, i32, i32,
                                      ctypes.POINTER(fe_schedule), vp]),
            "fe_batch_autotune": (i, [vp, ctypes.POINTER(fe_batch_item), i32, i32, i32, vp,
                                      ctypes.POINTER(fe_schedule), ctypes.POINTER(ctypes.c_float)]),
            "fe_batch_graph_create": (i, [vp, ctypes.POINTER(fe_batch_item), i32, i32, i32, i32,
                                          ctypes.POINTER(fe_schedule), vp, pp]),
            "fe_batch_tuned": (i, [vp, ctypes.POINTER(fe_batch_item), i32, i32, i32, ctypes.POINTER(fe_schedule)]),
            "fe_batch_graph_launch": (i, [vp, vp]),
            "fe_batch_graph_destroy": (i, [vp]),
            "fe_server_start": (i, [vp, i32, i32, ctypes.c_size_t, pp]),
            "fe_server_stop": (i, [vp]),
            "fe_batch_submit": (i, [vp, ctypes.POINTER(fe_request), i32, ctypes.POINTER(ctypes.c_uint64)]),
            "fe_poll": (i, [vp, ctypes.c_uint64, ctypes.POINTER(fe_result)]),
            "fe_wait": (i, [vp, ctypes.c_uint64, ctypes.c_double, ctypes.POINTER(fe_result)]),
            "fe_cancel": (i, [vp, ctypes.c_uint64]),
            "fe_release": (i, [vp, ctypes.c_uint64]),
            "fe_server_stats_get": (i, [vp, ctypes.POINTER(fe_server_stats)]),
            "fe_generate_scaled": (i, [vp, vp, i32, i64, ctypes.c_uint64, vp, vp]),
            "fe_server_timeline": (i, [vp, i64, i64, ctypes.POINTER(fe_span), ctypes.POINTER(i64)]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _check(rc, where):
    if rc != FE_OK:
        raise FeError(rc, where)


def _addr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        if not x.is_cuda:
            raise ValueError("expected a CUDA tensor")
        if not x.is_contiguous():
            raise ValueError("expected a contiguous tensor")
        return x.data_ptr()
    raise TypeError(f"cannot pass {type(x)} as a device pointer")


def _stream(s):
    if s is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(s, int):
        return s
    return s.cuda_stream


def fe_strerror(code: int) -> str:
    return load().fe_strerror(int(code)).decode()


def fe_last_cuda_error() -> str:
    return load().fe_last_cuda_error().decode()


def fe_kernel_launches() -> int:
    return int(load().fe_kernel_launches())


def fe_debug_checks() -> bool:
    return bool(load().fe_debug_checks())


def fe_device_status(ctx, stream=None) -> int:
    """First error recorded by a kernel since the last call (0 = none); clears it."""
    return int(load().fe_device_status(ctx, _stream(stream)))


def fe_tune_set(ctx, knob: int, value: int):
    _check(load().fe_tune_set(ctx, int(knob), int(value)), "fe_tune_set")


def fe_tune_get(ctx, knob: int) -> int:
    out = ctypes.c_int()
    _check(load().fe_tune_get(ctx, int(knob), ctypes.byref(out)), "fe_tune_get")
    return out.value


def fe_create(device: int = 0, hbm_budget_bytes: int = 0):
    out = ctypes.c_void_p()
    _check(load().fe_create(ctypes.byref(out), int(device), int(hbm_budget_bytes)), "fe_create")
    return out


def fe_create_ex(device: int = 0, hbm_budget_bytes: int = 0, pool_limit_bytes: int = 0):
    out = ctypes.c_void_p()
    _check(load().fe_create_ex(ctypes.byref(out), int(device), int(hbm_budget_bytes), int(pool_limit_bytes)),
           "fe_create_ex")
    return out


def fe_destroy(ctx):
    _check(load().fe_destroy(ctx), "fe_destroy")


def fe_pattern_build(ctx, n_elem, dofs_per_elem, n_dofs, elem_dofs, flags=FE_PATTERN_ALL, stream=None):
    if hasattr(elem_dofs, "dtype"):
        import torch
        if elem_dofs.dtype != torch.int32:
            raise TypeError("elem_dofs must be int32")
    out = ctypes.c_void_p()
    _check(load().fe_pattern_build(ctx, int(n_elem), int(dofs_per_elem), int(n_dofs), _addr(elem_dofs),
                                   int(flags), _stream(stream), ctypes.byref(out)), "fe_pattern_build")
    return out


def fe_pattern_csr_noalloc(n_elem, dofs_per_elem, n_dofs, elem_dofs, row_ptr, col_idx, col_capacity,
                           stream=None):
    """CSR pattern into caller-provided device buffers without allocating;
    returns nnz.  Raises FeError (code FE_ERR_INVALID_ARG) when col_capacity
    is below nnz; the error's .nnz then holds the size needed."""
    nnz = ctypes.c_int64()
    rc = load().fe_pattern_csr_noalloc(int(n_elem), int(dofs_per_elem), int(n_dofs), _addr(elem_dofs),
                                       _addr(row_ptr), _addr(col_idx), int(col_capacity), ctypes.byref(nnz),
                                       _stream(stream))
    if rc != FE_OK:
        err = FeError(rc, "fe_pattern_csr_noalloc")
        err.nnz = nnz.value
        raise err
    return nnz.value


def fe_pattern_free(pattern):
    _check(load().fe_pattern_free(pattern), "fe_pattern_free")


def fe_pattern_free_async(pattern, stream=None):
    _check(load().fe_pattern_free_async(pattern, _stream(stream)), "fe_pattern_free_async")


def fe_pattern_csr(pattern):
    rp, ci, nnz = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_int64()
    _check(load().fe_pattern_csr(pattern, ctypes.byref(rp), ctypes.byref(ci), ctypes.byref(nnz)), "fe_pattern_csr")
    return rp.value, ci.value, nnz.value


def fe_pattern_crac(pattern):
    rp, ca, n = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_int64()
    _check(load().fe_pattern_crac(pattern, ctypes.byref(rp), ctypes.byref(ca), ctypes.byref(n)), "fe_pattern_crac")
    return rp.value, ca.value, n.value


def fe_pattern_adjacency(pattern):
    blk, ap, a = ctypes.c_int32(), ctypes.c_void_p(), ctypes.c_void_p()
    _check(load().fe_pattern_adjacency(pattern, ctypes.byref(blk), ctypes.byref(ap), ctypes.byref(a)),
           "fe_pattern_adjacency")
    return blk.value, ap.value, a.value


def fe_pattern_info_get(pattern) -> dict:
    info = fe_pattern_info()
    _check(load().fe_pattern_info_get(pattern, ctypes.byref(info)), "fe_pattern_info_get")
    return {name: getattr(info, name) for name, _ in fe_pattern_info._fields_}


def fe_pattern_colour(ctx, pattern, stream=None) -> int:
    """Greedy first-fit element colouring on the device; returns the number of colours."""
    n = ctypes.c_int32()
    _check(load().fe_pattern_colour(ctx, pattern, _stream(stream), ctypes.byref(n)), "fe_pattern_colour")
    return n.value


def fe_pattern_colours(pattern):
    n, c = ctypes.c_int32(), ctypes.c_void_p()
    _check(load().fe_pattern_colours(pattern, ctypes.byref(n), ctypes.byref(c)), "fe_pattern_colours")
    return n.value, c.value


def fe_assemble_csr(ctx, pattern, elem_mats, values, mode=FE_ATOMIC, accumulate=0, stream=None):
    _check(load().fe_assemble_csr(ctx, pattern, _addr(elem_mats), _addr(values), int(mode), int(accumulate),
                                  _stream(stream)), "fe_assemble_csr")


def fe_assemble_crac(ctx, pattern, elem_mats, values, mode=FE_ATOMIC, accumulate=0, stream=None):
    _check(load().fe_assemble_crac(ctx, pattern, _addr(elem_mats), _addr(values), int(mode), int(accumulate),
                                   _stream(stream)), "fe_assemble_crac")


def fe_spmv_csr(ctx, pattern, values, x, y, stream=None):
    _check(load().fe_spmv_csr(ctx, pattern, _addr(values), _addr(x), _addr(y), _stream(stream)), "fe_spmv_csr")


def fe_spmv_crac(ctx, pattern, values, x, y, stream=None):
    _check(load().fe_spmv_crac(ctx, pattern, _addr(values), _addr(x), _addr(y), _stream(stream)), "fe_spmv_crac")


def _items(items):
    """items: sequence of (pattern handle or Pattern, K tensor/addr, values tensor/addr[, times tensor/addr])."""
    arr = (fe_batch_item * max(len(items), 1))()
    for k, item in enumerate(items):
        pat, K, v = item[:3]
        h = pat.handle if isinstance(pat, Pattern) else pat
        arr[k].pattern = h.value if isinstance(h, ctypes.c_void_p) else h
        arr[k].elem_mats = _addr(K)
        arr[k].values = _addr(v)
        arr[k].times_ns = _addr(item[3]) if len(item) > 3 else None
    return arr


def _sched(sched):
    if sched is None:
        return None
    kind, tile = sched
    return ctypes.byref(fe_schedule(int(kind), int(tile)))


def fe_assemble_batch(ctx, items, fmt=FE_FORMAT_CSR, mode=FE_ATOMIC, accumulate=0, sched=None, stream=None):
    arr = _items(items)
    _check(load().fe_assemble_batch(ctx, arr, len(items), int(fmt), int(mode), int(accumulate), _sched(sched),
                                    _stream(stream)), "fe_assemble_batch")


def fe_batch_autotune(ctx, items, fmt=FE_FORMAT_CSR, mode=FE_ATOMIC, stream=None):
    """-> (kind, tile, ms) of the fastest schedule; remembered for this batch signature."""
    arr = _items(items)
    best, ms = fe_schedule(), ctypes.c_float()
    _check(load().fe_batch_autotune(ctx, arr, len(items), int(fmt), int(mode), _stream(stream), ctypes.byref(best),
                                    ctypes.byref(ms)), "fe_batch_autotune")
    return best.kind, best.tile, ms.value


def fe_batch_tuned(ctx, items, fmt=FE_FORMAT_CSR, mode=FE_ATOMIC):
    """-> (kind, tile) that fe_assemble_batch takes for this batch signature,
    or None when no tuned schedule is known (in this context or the
    FEASM_TUNE_CACHE file)."""
    arr = _items(items)
    out = fe_schedule()
    rc = load().fe_batch_tuned(ctx, arr, len(items), int(fmt), int(mode), ctypes.byref(out))
    if rc == FE_ERR_NOT_FOUND:
        return None
    _check(rc, "fe_batch_tuned")
    return out.kind, out.tile


def fe_batch_graph_create(ctx, items, fmt=FE_FORMAT_CSR, mode=FE_ATOMIC, accumulate=0, sched=None, stream=None):
    arr = _items(items)
    out = ctypes.c_void_p()
    _check(load().fe_batch_graph_create(ctx, arr, len(items), int(fmt), int(mode), int(accumulate), _sched(sched),
                                        _stream(stream), ctypes.byref(out)), "fe_batch_graph_create")
    return out


def fe_batch_graph_launch(graph, stream=None):
    _check(load().fe_batch_graph_launch(graph, _stream(stream)), "fe_batch_graph_launch")


def fe_batch_graph_destroy(graph):
    _check(load().fe_batch_graph_destroy(graph), "fe_batch_graph_destroy")


def fe_server_start(ctx, n_streams=4, max_batch=64, hbm_budget_bytes=0):
    out = ctypes.c_void_p()
    _check(load().fe_server_start(ctx, int(n_streams), int(max_batch), int(hbm_budget_bytes), ctypes.byref(out)),
           "fe_server_start")
    return out


def fe_server_stop(server):
    _check(load().fe_server_stop(server), "fe_server_stop")


def make_request(pattern_key, elem_dofs, n_dofs, *, elem_mats=None, k_ref=None, seed=0, fmt=FE_FORMAT_CSR,
                 mode=FE_DETERMINISTIC, ready_event=None, deadline_s=0.0):
    """An fe_request for a device connectivity tensor [n_elem, n_loc]."""
    r = fe_request()
    r.pattern_key = int(pattern_key)
    r.n_elem = int(elem_dofs.shape[0])
    r.dofs_per_elem = int(elem_dofs.shape[1])
    r.format = int(fmt)
    r.n_dofs = int(n_dofs)
    r.elem_dofs = _addr(elem_dofs)
    r.elem_mats = _addr(elem_mats)
    r.k_ref = _addr(k_ref)
    r.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    r.mode = int(mode)
    r.ready_event = None if ready_event is None else int(ready_event.cuda_event)
    r.deadline_s = float(deadline_s)
    return r


def fe_batch_submit(server, requests):
    arr = (fe_request * max(len(requests), 1))(*requests)
    tickets = (ctypes.c_uint64 * max(len(requests), 1))()
    _check(load().fe_batch_submit(server, arr, len(requests), tickets), "fe_batch_submit")
    return [int(tickets[k]) for k in range(len(requests))]


def _result_dict(res):
    return {name: getattr(res, name) for name, _ in fe_result._fields_}


def fe_poll(server, ticket):
    res = fe_result()
    _check(load().fe_poll(server, int(ticket), ctypes.byref(res)), "fe_poll")
    return _result_dict(res)


def fe_wait(server, ticket, timeout_s=60.0):
    res = fe_result()
    _check(load().fe_wait(server, int(ticket), float(timeout_s), ctypes.byref(res)), "fe_wait")
    return _result_dict(res)


def fe_cancel(server, ticket):
    _check(load().fe_cancel(server, int(ticket)), "fe_cancel")


def fe_release(server, ticket):
    _check(load().fe_release(server, int(ticket)), "fe_release")


def fe_server_stats_get(server):
    st = fe_server_stats()
    _check(load().fe_server_stats_get(server, ctypes.byref(st)), "fe_server_stats_get")
    return {name: getattr(st, name) for name, _ in fe_server_stats._fields_}


def fe_server_timeline(server):
    """The server's device spans as a list of (start_ms, end_ms, stream,
    n_requests); stream -1 marks a pattern build."""
    n = ctypes.c_int64()
    _check(load().fe_server_timeline(server, 0, 0, None, ctypes.byref(n)), "fe_server_timeline")
    buf = (fe_span * max(n.value, 1))()
    _check(load().fe_server_timeline(server, 0, n.value, buf, ctypes.byref(n)), "fe_server_timeline")
    return [(buf[k].start_ms, buf[k].end_ms, buf[k].stream, buf[k].n_requests) for k in range(min(n.value, len(buf)))]


def fe_generate_scaled(ctx, k_ref, n_loc, n_elem, seed, out, stream=None):
    _check(load().fe_generate_scaled(ctx, _addr(k_ref), int(n_loc), int(n_elem), int(seed) & 0xFFFFFFFFFFFFFFFF,
                                     _addr(out), _stream(stream)), "fe_generate_scaled")


# ---- views of library-owned device arrays --------------------------------

class _DeviceArray:
    def __init__(self, ptr, n, typestr):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": typestr, "data": (int(ptr or 0), False),
                                         "version": 2, "strides": None}


def device_view(ptr, n, dtype):
    """A torch CUDA tensor aliasing n elements at a library-owned address."""
    import torch
    typestr = {torch.int64: "<i8", torch.int32: "<i4", torch.uint32: "<u4", torch.float64: "<f8",
               torch.uint8: "|u1"}[dtype]
    if n == 0:
        return torch.empty(0, dtype=dtype, device="cuda")
    return torch.as_tensor(_DeviceArray(ptr, n, typestr), device="cuda")


class Pattern:
    """Owns an fe_pattern handle; exposes its arrays as torch views."""

    def __init__(self, ctx, elem_dofs, n_dofs, flags=FE_PATTERN_ALL, stream=None):
        n_e, n_loc = elem_dofs.shape
        self.ctx = ctx
        self.handle = fe_pattern_build(ctx, n_e, n_loc, n_dofs, elem_dofs, flags, stream)
        self.info = fe_pattern_info_get(self.handle)

    def csr(self):
        import torch
        rp, ci, nnz = fe_pattern_csr(self.handle)
        return device_view(rp, self.info["n_dofs"] + 1, torch.int64), device_view(ci, nnz, torch.int32)

    def crac(self):
        import torch
        rp, ca, n = fe_pattern_crac(self.handle)
        return device_view(rp, self.info["n_dofs"] + 1, torch.int64), device_view(ca, n, torch.int32)

    def adjacency(self):
        """(B, adj_ptr [n_dofs/B + 1], adj [n_elem * n_loc / B]) as torch views."""
        import torch
        blk, ap, a = fe_pattern_adjacency(self.handle)
        n_inc = self.info["n_elem"] * self.info["n_loc"] // blk
        return blk, device_view(ap, self.info["n_dofs"] // blk + 1, torch.int64), device_view(a, n_inc, torch.int32)

    def free(self):
        if self.handle is not None:
            fe_pattern_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass
