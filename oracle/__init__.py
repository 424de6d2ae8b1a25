"""CPU oracle for finite-element sparse-matrix assembly (arXiv 2012.00585).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by
the benchmark's CPU-baseline / reference leg, never by the CUDA product path.
It shares no code with ``paper_2012_00585_gb300``.

The arithmetic lives in ``oracle.c`` (plain serial C, one function per
definition or algorithm of the paper, each citing its passage); this module
compiles it with gcc on first use and wraps it with numpy arrays.

Pins (what checks the oracle against something other than itself) are in
``tests/test_oracle_pins.py``.  Parity status per function:
  csr_pattern, csr_lookup, assemble_csr, crac_from_csr, crac_lookup,
  compress_dofs, assemble_crac, greedy_colouring, spmv_csr, spmv_crac: pinned.
"""

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None
_lock = threading.Lock()

OR_ERRORS = {
    -1: "invalid argument",
    -2: "DOF out of range",
    -3: "duplicate DOF inside an element",
    -4: "entry not in pattern",
    -5: "out of memory",
}


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    """Compile oracle.c into _build/liboracle.so (gcc, -O2 -ffp-contract=off)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        i64, i32, vp = ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p
        sig = {
            "or_check_elements": (ctypes.c_int, [i64, i32, i64, vp]),
            "or_csr_pattern": (i64, [i64, i32, i64, vp, vp, ctypes.POINTER(vp)]),
            "or_csr_lookup": (i64, [vp, vp, i64, i32]),
            "or_assemble_csr": (ctypes.c_int, [i64, i32, vp, vp, vp, vp, vp, vp]),
            "or_crac_from_csr": (i64, [i64, i64, vp, vp, vp, ctypes.POINTER(vp)]),
            "or_crac_lookup": (i64, [vp, vp, i64, i32]),
            "or_compress_dofs": (i32, [i32, vp, vp]),
            "or_assemble_crac": (ctypes.c_int, [i64, i32, vp, vp, vp, vp, vp, vp]),
            "or_greedy_colouring": (i32, [i64, i32, i64, vp, vp]),
            "or_spmv_csr": (None, [i64, vp, vp, vp, vp, vp]),
            "or_spmv_crac": (None, [i64, vp, vp, vp, vp, vp]),
            "or_free": (None, [vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _check(rc):
    if rc < 0:
        raise OracleError(OR_ERRORS.get(int(rc), f"error {rc}"))
    return rc


def check_elements(elem_dofs, n_dofs):
    D = _c(elem_dofs, np.int32)
    n_e, n_loc = D.shape
    return _check(_load().or_check_elements(n_e, n_loc, n_dofs, _ptr(D)))


def csr_pattern(elem_dofs, n_dofs):
    """(row_ptr int64 [n_dofs+1], col_idx int32 [nnz]) -- §2.2 CSR pattern."""
    lib = _load()
    D = _c(elem_dofs, np.int32)
    n_e, n_loc = D.shape
    row_ptr = np.zeros(n_dofs + 1, dtype=np.int64)
    out = ctypes.c_void_p()
    nnz = _check(lib.or_csr_pattern(n_e, n_loc, n_dofs, _ptr(D), _ptr(row_ptr), ctypes.byref(out)))
    try:
        buf = (ctypes.c_int32 * max(nnz, 1)).from_address(out.value)
        col_idx = np.frombuffer(buf, dtype=np.int32, count=nnz).copy()
    finally:
        lib.or_free(out)
    return row_ptr, col_idx


def csr_lookup(row_ptr, col_idx, i, j):
    return int(_load().or_csr_lookup(_ptr(row_ptr), _ptr(col_idx), int(i), int(j)))


def assemble_csr(elem_dofs, K, row_ptr, col_idx, values=None, order=None):
    """Listing 2 into a CSR values array (zeroed unless ``values`` is given)."""
    D = _c(elem_dofs, np.int32)
    n_e, n_loc = D.shape
    Kc = _c(K, np.float64).reshape(n_e, n_loc, n_loc)
    rp = _c(row_ptr, np.int64)
    ci = _c(col_idx, np.int32)
    v = np.zeros(ci.shape[0], dtype=np.float64) if values is None else _c(values, np.float64).copy()
    o = None if order is None else _c(order, np.int64)
    _check(_load().or_assemble_csr(n_e, n_loc, _ptr(D), _ptr(Kc), _ptr(rp), _ptr(ci), _ptr(v), _ptr(o)))
    return v


def crac_from_csr(row_ptr, col_idx, n_cols):
    """(crac_ptr int64 [n_rows+1], col_align int32 [n_ca]) -- §2.2 CRAC, Fig. 1d."""
    lib = _load()
    rp = _c(row_ptr, np.int64)
    ci = _c(col_idx, np.int32)
    n_rows = rp.shape[0] - 1
    crac_ptr = np.zeros(n_rows + 1, dtype=np.int64)
    out = ctypes.c_void_p()
    n_ca = _check(lib.or_crac_from_csr(n_rows, n_cols, _ptr(rp), _ptr(ci), _ptr(crac_ptr), ctypes.byref(out)))
    try:
        buf = (ctypes.c_int32 * n_ca).from_address(out.value)
        col_align = np.frombuffer(buf, dtype=np.int32, count=n_ca).copy()
    finally:
        lib.or_free(out)
    return crac_ptr, col_align


def crac_lookup(crac_ptr, col_align, i, c):
    return int(_load().or_crac_lookup(_ptr(crac_ptr), _ptr(col_align), int(i), int(c)))


def compress_dofs(dofs):
    d = _c(dofs, np.int32)
    out = np.zeros(2 * max(d.shape[0], 1), dtype=np.int32)
    n = _load().or_compress_dofs(d.shape[0], _ptr(d), _ptr(out))
    return out[:n].copy()


def assemble_crac(elem_dofs, K, crac_ptr, col_align, nnz, values=None, order=None):
    """Listing 5's arithmetic, serial, into the CRAC values array."""
    D = _c(elem_dofs, np.int32)
    n_e, n_loc = D.shape
    Kc = _c(K, np.float64).reshape(n_e, n_loc, n_loc)
    cp = _c(crac_ptr, np.int64)
    ca = _c(col_align, np.int32)
    v = np.zeros(nnz, dtype=np.float64) if values is None else _c(values, np.float64).copy()
    o = None if order is None else _c(order, np.int64)
    _check(_load().or_assemble_crac(n_e, n_loc, _ptr(D), _ptr(Kc), _ptr(cp), _ptr(ca), _ptr(v), _ptr(o)))
    return v


def greedy_colouring(elem_dofs, n_dofs):
    """(n_colours, colour int32 [n_e]) -- greedy colouring used by Listing 6."""
    D = _c(elem_dofs, np.int32)
    n_e, n_loc = D.shape
    colour = np.zeros(n_e, dtype=np.int32)
    k = _check(_load().or_greedy_colouring(n_e, n_loc, n_dofs, _ptr(D), _ptr(colour)))
    return int(k), colour


def spmv_csr(row_ptr, col_idx, values, x):
    rp = _c(row_ptr, np.int64)
    ci = _c(col_idx, np.int32)
    v = _c(values, np.float64)
    xx = _c(x, np.float64)
    y = np.zeros(rp.shape[0] - 1, dtype=np.float64)
    _load().or_spmv_csr(rp.shape[0] - 1, _ptr(rp), _ptr(ci), _ptr(v), _ptr(xx), _ptr(y))
    return y


def spmv_crac(crac_ptr, col_align, values, x):
    cp = _c(crac_ptr, np.int64)
    ca = _c(col_align, np.int32)
    v = _c(values, np.float64)
    xx = _c(x, np.float64)
    y = np.zeros(cp.shape[0] - 1, dtype=np.float64)
    _load().or_spmv_crac(cp.shape[0] - 1, _ptr(cp), _ptr(ca), _ptr(v), _ptr(xx), _ptr(y))
    return y


def assemble(elem_dofs, K, n_dofs, order=None):
    """Convenience: pattern + values by Listing 2 -> (row_ptr, col_idx, values)."""
    row_ptr, col_idx = csr_pattern(elem_dofs, n_dofs)
    return row_ptr, col_idx, assemble_csr(elem_dofs, K, row_ptr, col_idx, order=order)
