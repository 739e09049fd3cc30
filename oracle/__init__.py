"""FP64 CPU oracle for sparse MTTKRP along every mode and for CPD-ALS.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The CUDA library and
its Python binding never import this package, and this package imports
nothing from them.

The arithmetic lives in ``oracle.c`` (plain C, FP64, no blocking or fusion);
this module compiles it with gcc on first use and marshals numpy arrays.

Which passage each routine follows:

* :func:`mttkrp` / :func:`mttkrp_rows` -- Sec. II-A6 (elementwise
  computation) generalised to N modes as in Algorithm 2; the output of Eq. 1
  is a fresh matrix.  :func:`mttkrp_omp` evaluates the same definition on all
  host cores (thread-private outputs summed at the end) for the CPU baseline.
* :func:`mode_permutation` -- Sec. III-B2 (nonzeros ordered by the output-mode
  index); ties by the other modes in ascending mode order, then by position.
* :func:`partition_equal` -- Sec. III-B2 (kappa equal-size partitions).
* :func:`partition_balanced` -- a design choice of this library, not a rule
  of the paper: Sec. III-B2's ordered nonzeros cut into equal-cost work
  units (nonzeros plus a charge per output-row start).
* :func:`units_from_partitions` -- the equal split of each partition into
  work units that the SCHEME1/SCHEME2 policies use (also a design choice).
* :func:`partition_scheme1` -- Sec. III-B1 (degree-ordered cyclic deal).
* :func:`adaptive_policy` -- Sec. III-B (I_d >= kappa selects Scheme 1).
* :func:`cpd_als` -- Sec. II-A5 (CP-ALS over Eq. 1), standard normal-equation
  update and fit.

Every routine is pinned by ``tests/test_oracle_pins.py`` against brute force,
closed forms and invariants that do not go through this code.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT_DIR = os.path.join(_HERE, "_lib")
_SO = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, ERR_ARG, ERR_INDEX, ERR_NOMEM, ERR_NUMERIC = 0, 1, 2, 3, 5

PREC = {"fp64": 0, "fp32": 1, "bf16": 2}


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_lib/liboracle.so (gcc -O2)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(_SRC)):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC",
                           "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _SO)
    return _SO


_SO_OMP = os.path.join(_OUT_DIR, "liboracle_omp.so")
_lib_omp = None


def build_omp(force: bool = False) -> str:
    """Compile oracle.c with -fopenmp into oracle/_lib/liboracle_omp.so (the
    all-core CPU baseline; raises OracleError when OpenMP is unavailable)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_SO_OMP)
            and os.path.getmtime(_SO_OMP) >= os.path.getmtime(_SRC)):
        return _SO_OMP
    tmp = _SO_OMP + f".tmp{os.getpid()}"
    res = subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-shared", "-fPIC",
                          "-o", tmp, _SRC, "-lm"], capture_output=True, text=True)
    if res.returncode != 0:
        raise OracleError("OpenMP build of the oracle failed: " + res.stderr.strip()[-300:])
    os.replace(tmp, _SO_OMP)
    return _SO_OMP


def _load_omp():
    global _lib_omp
    with _lock:
        if _lib_omp is None:
            lib = ctypes.CDLL(build_omp())
            P = ctypes.c_void_p
            i64, i32 = ctypes.c_int64, ctypes.c_int
            lib.oracle_mttkrp_omp.argtypes = [i32, P, i64, P, P, i32, P, i32, i32, P, P]
            _lib_omp = lib
    return _lib_omp


def mttkrp_omp(dims, idx, vals, factors, mode, threads=0):
    """M_mode by the same definition on `threads` OpenMP threads (0 = all)
    with thread-private outputs added in thread order.  Returns (M, threads
    used).  The all-core CPU baseline; not used as a parity reference."""
    lib = _load_omp()
    idx = _idx_list(idx)
    vals = _f64(vals)
    fac = [_f64(f) for f in factors]
    R = fac[0].shape[1]
    dims_a = np.asarray(dims, dtype=np.int64)
    out = np.empty((int(dims[mode]), R), dtype=np.float64)
    used = ctypes.c_int(0)
    _check(lib.oracle_mttkrp_omp(len(idx), dims_a.ctypes.data, int(vals.size),
                                 _ptr_array(idx), vals.ctypes.data, R, _ptr_array(fac),
                                 int(mode), int(threads), out.ctypes.data,
                                 ctypes.addressof(used)),
           "oracle_mttkrp_omp")
    return out, int(used.value)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i64, i32 = ctypes.c_int64, ctypes.c_int
            lib.oracle_mttkrp.argtypes = [i32, P, i64, P, P, i32, P, i32, P]
            lib.oracle_mttkrp_rows.argtypes = [i32, P, i64, P, P, i32, P, i32,
                                               i64, P, P]
            lib.oracle_mode_permutation.argtypes = [i32, i64, P, i32, P]
            lib.oracle_partition_equal.argtypes = [i64, i32, P]
            lib.oracle_partition_balanced.argtypes = [i64, P, i64, i64, P]
            lib.oracle_partition_scheme1.argtypes = [i32, P, i64, P, i32, i32,
                                                     P, P, P]
            lib.oracle_cpd_als.argtypes = [i32, P, i64, P, P, i32, P, i32, i32,
                                           P, P]
            lib.oracle_norm2.argtypes = [i32, i64, P, P, P]
            lib.oracle_als_update.argtypes = [i32, P, i32, P, i32, P, i32, P]
            lib.oracle_store_round.argtypes = [ctypes.c_double, i32]
            lib.oracle_store_round.restype = ctypes.c_double
            lib.oracle_store_round_array.argtypes = [P, i64, i32]
            _lib = lib
    return _lib


def _check(rc: int, what: str):
    if rc != OK:
        raise OracleError(f"{what} failed with oracle status {rc}")


def _ptr_array(arrays):
    arr = (ctypes.c_void_p * len(arrays))(*[a.ctypes.data for a in arrays])
    return arr


def _idx_list(idx):
    return [np.ascontiguousarray(a, dtype=np.int32) for a in idx]


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def mttkrp(dims, idx, vals, factors, mode):
    """M_mode (I_mode x R, FP64) by the elementwise definition."""
    lib = _load()
    idx = _idx_list(idx)
    vals = _f64(vals)
    fac = [_f64(f) for f in factors]
    R = fac[0].shape[1]
    dims_a = np.asarray(dims, dtype=np.int64)
    out = np.empty((int(dims[mode]), R), dtype=np.float64)
    _check(lib.oracle_mttkrp(len(idx), dims_a.ctypes.data, int(vals.size),
                             _ptr_array(idx), vals.ctypes.data, R,
                             _ptr_array(fac), int(mode), out.ctypes.data),
           "oracle_mttkrp")
    return out


def mttkrp_rows(dims, idx, vals, factors, mode, rows):
    """Rows `rows` of M_mode (len(rows) x R, FP64) by the same definition."""
    lib = _load()
    idx = _idx_list(idx)
    vals = _f64(vals)
    fac = [_f64(f) for f in factors]
    R = fac[0].shape[1]
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    dims_a = np.asarray(dims, dtype=np.int64)
    out = np.empty((rows.size, R), dtype=np.float64)
    _check(lib.oracle_mttkrp_rows(len(idx), dims_a.ctypes.data, int(vals.size),
                                  _ptr_array(idx), vals.ctypes.data, R,
                                  _ptr_array(fac), int(mode), int(rows.size),
                                  rows.ctypes.data, out.ctypes.data),
           "oracle_mttkrp_rows")
    return out


def mode_permutation(idx, mode):
    """Input positions of the nonzeros in the mode-`mode` copy order (int64)."""
    lib = _load()
    idx = _idx_list(idx)
    nnz = idx[0].size
    perm = np.empty(nnz, dtype=np.int64)
    _check(lib.oracle_mode_permutation(len(idx), nnz, _ptr_array(idx),
                                       int(mode), perm.ctypes.data),
           "oracle_mode_permutation")
    return perm


def partition_equal(nnz, kappa):
    """Scheme 2 offsets floor(z*nnz/kappa), z = 0..kappa (int64)."""
    lib = _load()
    off = np.empty(int(kappa) + 1, dtype=np.int64)
    _check(lib.oracle_partition_equal(int(nnz), int(kappa), off.ctypes.data),
           "oracle_partition_equal")
    return off


def partition_balanced(idx, mode, parts, row_cost=16, perm=None):
    """Cost-balanced work-unit offsets (int64[parts+1]) of the mode copy:
    a nonzero costs 1 plus `row_cost` if it starts its output row."""
    lib = _load()
    idx = _idx_list(idx)
    if perm is None:
        perm = mode_permutation(idx, mode)
    rows = np.ascontiguousarray(idx[mode][perm], dtype=np.int32)
    off = np.empty(int(parts) + 1, dtype=np.int64)
    _check(lib.oracle_partition_balanced(int(rows.size), rows.ctypes.data, int(parts),
                                         int(row_cost), off.ctypes.data),
           "oracle_partition_balanced")
    return off


def partition_balanced_rows(rows_sorted, parts, row_cost=16):
    """The same work units from the output-mode indices in copy order (the
    partition depends only on that non-decreasing sequence)."""
    lib = _load()
    rows = np.ascontiguousarray(rows_sorted, dtype=np.int32)
    off = np.empty(int(parts) + 1, dtype=np.int64)
    _check(lib.oracle_partition_balanced(int(rows.size), rows.ctypes.data, int(parts),
                                         int(row_cost), off.ctypes.data),
           "oracle_partition_balanced")
    return off


def units_from_partitions(off, units):
    """Work units of a partition vector: unit w of partition z starts at
    off[z] + floor((off[z+1] - off[z]) * w / units)."""
    off = np.asarray(off, dtype=np.int64)
    out = []
    for z in range(off.size - 1):
        for w in range(units):
            out.append(off[z] + ((off[z + 1] - off[z]) * w) // units)
    out.append(off[-1])
    return np.asarray(out, dtype=np.int64)


def partition_scheme1(dims, idx, mode, kappa):
    """Scheme 1: (perm int64[nnz], offsets int64[kappa+1], row_part int32[I])."""
    lib = _load()
    idx = _idx_list(idx)
    nnz = idx[0].size
    dims_a = np.asarray(dims, dtype=np.int64)
    perm = np.empty(nnz, dtype=np.int64)
    off = np.empty(int(kappa) + 1, dtype=np.int64)
    row_part = np.empty(int(dims[mode]), dtype=np.int32)
    _check(lib.oracle_partition_scheme1(len(idx), dims_a.ctypes.data, nnz,
                                        _ptr_array(idx), int(mode), int(kappa),
                                        perm.ctypes.data, off.ctypes.data,
                                        row_part.ctypes.data),
           "oracle_partition_scheme1")
    return perm, off, row_part


def adaptive_policy(dim, kappa):
    """Sec. III-B: Scheme 1 when I_d >= kappa, else Scheme 2."""
    return 1 if int(dim) >= int(kappa) else 2


def norm2(idx, vals):
    """|X|^2 with duplicate coordinates summed first."""
    lib = _load()
    idx = _idx_list(idx)
    vals = _f64(vals)
    out = ctypes.c_double(0.0)
    _check(lib.oracle_norm2(len(idx), int(vals.size), _ptr_array(idx),
                            vals.ctypes.data, ctypes.addressof(out)),
           "oracle_norm2")
    return out.value


def store_round(x, prec):
    """Storage rounding (prec 'fp64' | 'fp32' | 'bf16') of a scalar or array.

    FP32 is round-to-nearest-even from FP64; BF16 rounds that FP32 value to
    nearest even on its bit pattern.  Returns FP64 values."""
    lib = _load()
    if np.isscalar(x):
        return lib.oracle_store_round(float(x), PREC[prec])
    a = np.array(x, dtype=np.float64, copy=True, order="C")
    lib.oracle_store_round_array(a.ctypes.data, int(a.size), PREC[prec])
    return a


def als_update(dims, factors, mode, M, prec="fp64"):
    """One CP-ALS factor update of `mode` from its MTTKRP result M.

    Returns (new factor list (FP64, the updated one rounded to `prec`),
    lambda FP64[R]).  Raises OracleError(status 5) if the Hadamard product of
    the other Grams is not positive definite."""
    lib = _load()
    fac = [_f64(f).copy() for f in factors]
    M = _f64(M)
    R = fac[0].shape[1]
    dims_a = np.asarray(dims, dtype=np.int64)
    lam = np.zeros(R, dtype=np.float64)
    _check(lib.oracle_als_update(len(fac), dims_a.ctypes.data, R,
                                 _ptr_array(fac), int(mode), M.ctypes.data,
                                 PREC[prec], lam.ctypes.data),
           "oracle_als_update")
    return fac, lam


def cpd_als(dims, idx, vals, factors, sweeps, prec="fp32"):
    """CP-ALS sweeps from the given initial factors.

    Returns (factors_out list of FP64 arrays, lambda FP64[R], fit FP64[sweeps]).
    The initial factors are first rounded to the storage precision `prec`.
    """
    lib = _load()
    idx = _idx_list(idx)
    vals = _f64(vals)
    fac = [_f64(f).copy() for f in factors]
    p = PREC[prec]
    if p:
        fac = [store_round(f, prec) for f in fac]
    R = fac[0].shape[1]
    dims_a = np.asarray(dims, dtype=np.int64)
    lam = np.zeros(R, dtype=np.float64)
    fit = np.zeros(max(int(sweeps), 1), dtype=np.float64)
    _check(lib.oracle_cpd_als(len(idx), dims_a.ctypes.data, int(vals.size),
                              _ptr_array(idx), vals.ctypes.data, R,
                              _ptr_array(fac), int(sweeps), p,
                              lam.ctypes.data, fit.ctypes.data),
           "oracle_cpd_als")
    return fac, lam, fit[:int(sweeps)]
