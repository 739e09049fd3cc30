"""Thin ctypes binding of the C ABI in include/spmttkrp.h.

Argument marshalling only: every computation runs in the CUDA library
(_lib/libspmttkrp.so).  There is no fallback of any kind -- if the library is
missing, :func:`load` raises.  PyTorch supplies device memory and the current
stream; the functions below keep the C names and argument order.
"""
from __future__ import annotations

import ctypes
import os

from . import _build

SPM_OK = 0
STATUS = {0: "SPM_OK", 1: "SPM_ERR_INVALID_ARG", 2: "SPM_ERR_INDEX_OUT_OF_RANGE",
          3: "SPM_ERR_OOM", 4: "SPM_ERR_CUDA", 5: "SPM_ERR_NUMERIC",
          6: "SPM_ERR_TIMEOUT", 7: "SPM_ERR_UNSUPPORTED"}

SPM_FACTOR_FP32 = 0x0
SPM_FACTOR_BF16 = 0x1
SPM_POLICY_BALANCED = 0 << 4
SPM_POLICY_SCHEME2 = 1 << 4
SPM_POLICY_SCHEME1 = 2 << 4
SPM_POLICY_ADAPTIVE = 3 << 4
SPM_ROW_COST = 16


SPM_PLAN_LEAN = 1 << 8
SPM_PLAN_FIBRE = 1 << 9


def SPM_UNITS_PER_PARTITION(R: int) -> int:
    u = 4096 // int(R)
    return 16 if u < 16 else (128 if u > 128 else u)
SPM_MAX_MODES = 7
SPM_MAX_RANK = 256


SPM_PARTITIONS_PER_SM = 2


def default_kappa() -> int:
    """Partition count of a plan made with SPM_KAPPA(0)."""
    return SPM_PARTITIONS_PER_SM * spm_device_sm_count()


def SPM_KAPPA(k: int) -> int:
    return (int(k) & 0xFFFF) << 16


class SpmError(RuntimeError):
    def __init__(self, status: int, what: str, text: str = ""):
        self.status = status
        super().__init__(f"{what}: {STATUS.get(status, status)} ({text})")


_lib = None

#: exported symbols declared in include/spmttkrp.h
SYMBOLS = ("spmttkrp_plan", "spmttkrp_plan_bytes", "spmttkrp_plan_permutation",
           "spmttkrp_plan_partition", "spmttkrp_plan_work_units", "spmttkrp_plan_scheme",
           "spmttkrp_plan_destroy", "spmttkrp_run", "cpd_als_step",
           "spmttkrp_plan_status", "spm_status_string", "spm_device_sm_count",
           "spmttkrp_run_noalloc", "spmttkrp_plan_repartition", "spmttkrp_plan_autotune",
           "spm_batch_create", "spm_batch_sweep",
           "spm_batch_status", "spm_batch_destroy", "spm_batch_autotune",
           "spmttkrp_plan_bytes_estimate", "spm_server_create", "spm_server_submit",
           "spm_server_step", "spm_server_job", "spm_server_result", "spm_server_usage",
           "spm_server_destroy", "spm_selftest_wait_timeout", "spm_inject_alloc_failure",
           "cpd_als_reset", "spm_server_snapshot", "spm_server_resume",
           "spmttkrp_run_all_host", "spm_selftest_mttkrp_timeout", "spmttkrp_noalloc_status",
           "spmttkrp_plan_fibre_count", "spm_selftest_tc_rowpass")


def library_path() -> str:
    return _build.so_path()


def load(build_if_missing: bool = False):
    """Load libspmttkrp.so (building it first only if asked).  Raises if the
    library is absent: the package has no other implementation."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(
                f"CUDA library {path} is missing; run __graft_entry__.build() "
                "(or python -m paper_2503_18198_gb300._build) first")
        path = _build.build()
    lib = ctypes.CDLL(path)
    P, i32, i64, u32 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint32
    lib.spmttkrp_plan.argtypes = [P, i32, P, i64, P, P, i32, u32, P]
    lib.spmttkrp_plan.restype = i32
    lib.spmttkrp_plan_bytes.argtypes = [P, P]
    lib.spmttkrp_plan_bytes.restype = i32
    lib.spmttkrp_plan_permutation.argtypes = [P, i32, P, P]
    lib.spmttkrp_plan_permutation.restype = i32
    lib.spmttkrp_plan_partition.argtypes = [P, i32, P, P, P]
    lib.spmttkrp_plan_partition.restype = i32
    lib.spmttkrp_plan_work_units.argtypes = [P, i32, P, P]
    lib.spmttkrp_plan_work_units.restype = i32
    lib.spmttkrp_plan_scheme.argtypes = [P, i32, P]
    lib.spmttkrp_plan_scheme.restype = i32
    lib.spmttkrp_plan_destroy.argtypes = [P]
    lib.spmttkrp_plan_destroy.restype = None
    lib.spmttkrp_run.argtypes = [P, i32, P, P, P]
    lib.spmttkrp_run.restype = i32
    lib.cpd_als_step.argtypes = [P, P, P, P, P]
    lib.cpd_als_step.restype = i32
    lib.spmttkrp_plan_status.argtypes = [P, P]
    lib.spmttkrp_plan_status.restype = i32
    lib.spm_status_string.argtypes = [i32]
    lib.spm_status_string.restype = ctypes.c_char_p
    lib.spmttkrp_run_noalloc.argtypes = [i32, P, i64, i32, i32, P, P, u32, P, P]
    lib.spmttkrp_run_noalloc.restype = i32
    lib.spmttkrp_plan_autotune.argtypes = [P, P, P, i32, i32, P, P, P]
    lib.spmttkrp_plan_autotune.restype = i32
    lib.spmttkrp_plan_repartition.argtypes = [P, i32, P]
    lib.spmttkrp_plan_repartition.restype = i32
    lib.spm_batch_create.argtypes = [P, i32, P, P, P, P, ctypes.c_double, i32, P]
    lib.spm_batch_create.restype = i32
    lib.spm_batch_sweep.argtypes = [P, P]
    lib.spm_batch_sweep.restype = i32
    lib.spm_batch_status.argtypes = [P, P, P, P]
    lib.spm_batch_status.restype = i32
    lib.spm_batch_autotune.argtypes = [i32, P, P, P, i32, i32, P, P, P]
    lib.spm_batch_autotune.restype = i32
    lib.spmttkrp_plan_bytes_estimate.argtypes = [i32, P, i64, i32, u32, P, P]
    lib.spmttkrp_plan_bytes_estimate.restype = i32
    lib.spm_server_create.argtypes = [P, ctypes.c_size_t, i32, u32, i64]
    lib.spm_server_create.restype = i32
    lib.spm_server_submit.argtypes = [P, P, P]
    lib.spm_server_submit.restype = i32
    lib.spm_server_step.argtypes = [P, P, P]
    lib.spm_server_step.restype = i32
    lib.spm_server_job.argtypes = [P, i64, P]
    lib.spm_server_job.restype = i32
    lib.spm_server_result.argtypes = [P, i64, P, P, P]
    lib.spm_server_result.restype = i32
    lib.spm_server_usage.argtypes = [P, P, P]
    lib.spm_server_usage.restype = i32
    lib.spm_server_destroy.argtypes = [P]
    lib.spm_server_destroy.restype = None
    lib.spm_selftest_wait_timeout.argtypes = [u32, P]
    lib.spm_selftest_wait_timeout.restype = i32
    lib.spm_selftest_mttkrp_timeout.argtypes = [P, i32, P, P, P]
    lib.spm_selftest_mttkrp_timeout.restype = i32
    lib.spmttkrp_plan_fibre_count.argtypes = [P, i32, P]
    lib.spmttkrp_plan_fibre_count.restype = i32
    lib.spm_selftest_tc_rowpass.argtypes = [i32, i64, P, P, P, P, P, P, P]
    lib.spm_selftest_tc_rowpass.restype = i32
    lib.spmttkrp_noalloc_status.argtypes = [P]
    lib.spmttkrp_noalloc_status.restype = i32
    lib.spm_inject_alloc_failure.argtypes = [i32]
    lib.spm_inject_alloc_failure.restype = None
    lib.spmttkrp_run_all_host.argtypes = [P, P, P, P]
    lib.spmttkrp_run_all_host.restype = i32
    lib.cpd_als_reset.argtypes = [P]
    lib.cpd_als_reset.restype = i32
    lib.spm_server_snapshot.argtypes = [P, i64, P, P, P, P, P]
    lib.spm_server_snapshot.restype = i32
    lib.spm_server_resume.argtypes = [P, P, i32, ctypes.c_double, P]
    lib.spm_server_resume.restype = i32
    lib.spm_batch_destroy.argtypes = [P]
    lib.spm_batch_destroy.restype = None
    lib.spm_device_sm_count.argtypes = []
    lib.spm_device_sm_count.restype = i32
    _lib = lib
    return lib


def _check(status: int, what: str):
    if status != SPM_OK:
        text = load().spm_status_string(status).decode()
        raise SpmError(status, what, text)


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _ptrs(tensors):
    return (ctypes.c_void_p * len(tensors))(
        *[t.data_ptr() if t is not None else 0 for t in tensors])


class Plan:
    """Owns an spmttkrp_plan_t; destroyed with the object or by destroy()."""

    def __init__(self, handle: ctypes.c_void_p, nmodes: int, dims, nnz: int,
                 rank: int, flags: int):
        self.handle = handle
        self.nmodes = nmodes
        self.dims = tuple(int(d) for d in dims)
        self.nnz = int(nnz)
        self.rank = int(rank)
        self.flags = int(flags)

    @property
    def bf16(self) -> bool:
        return bool(self.flags & SPM_FACTOR_BF16)

    def destroy(self):
        if self.handle:
            load().spmttkrp_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def spm_device_sm_count() -> int:
    return int(load().spm_device_sm_count())


def spm_status_string(status: int) -> str:
    return load().spm_status_string(int(status)).decode()


def spmttkrp_plan(dims, idx, vals, rank: int, flags: int = 0, stream=None) -> Plan:
    """idx: N int32 CUDA tensors [nnz]; vals: float32 CUDA tensor [nnz]."""
    lib = load()
    N = len(dims)
    nnz = int(vals.numel())
    dims_a = (ctypes.c_int64 * N)(*[int(d) for d in dims])
    handle = ctypes.c_void_p()
    st = lib.spmttkrp_plan(ctypes.byref(handle), N, dims_a, nnz, _ptrs(list(idx)),
                           ctypes.c_void_p(vals.data_ptr() if nnz else 0), int(rank),
                           int(flags) & 0xFFFFFFFF, _stream(stream))
    _check(st, "spmttkrp_plan")
    return Plan(handle, N, dims, nnz, rank, flags)


def spmttkrp_plan_bytes(plan: Plan) -> int:
    out = ctypes.c_size_t(0)
    _check(load().spmttkrp_plan_bytes(plan.handle, ctypes.byref(out)), "spmttkrp_plan_bytes")
    return int(out.value)


def spmttkrp_plan_permutation(plan: Plan, mode: int, perm, stream=None):
    """perm: int64 CUDA tensor [nnz], filled in copy order."""
    _check(load().spmttkrp_plan_permutation(plan.handle, int(mode),
                                            ctypes.c_void_p(perm.data_ptr() if plan.nnz else 0),
                                            _stream(stream)),
           "spmttkrp_plan_permutation")
    return perm


def spmttkrp_plan_partition(plan: Plan, mode: int, off, stream=None) -> int:
    """off: int64 CUDA tensor [kappa+1].  Returns kappa."""
    kappa = ctypes.c_int(0)
    _check(load().spmttkrp_plan_partition(plan.handle, int(mode),
                                          ctypes.c_void_p(off.data_ptr()),
                                          ctypes.byref(kappa), _stream(stream)),
           "spmttkrp_plan_partition")
    return int(kappa.value)


def spmttkrp_plan_work_units(plan: Plan, mode: int, off, stream=None):
    """off: int64 CUDA tensor [kappa*SPM_UNITS_PER_PARTITION(rank)+1]."""
    _check(load().spmttkrp_plan_work_units(plan.handle, int(mode), ctypes.c_void_p(off.data_ptr()),
                                           _stream(stream)),
           "spmttkrp_plan_work_units")
    return off


def spmttkrp_plan_scheme(plan: Plan, mode: int) -> int:
    out = ctypes.c_int(0)
    _check(load().spmttkrp_plan_scheme(plan.handle, int(mode), ctypes.byref(out)),
           "spmttkrp_plan_scheme")
    return int(out.value)


def spmttkrp_plan_repartition(plan: Plan, kappa: int, stream=None):
    """Recompute the partitions for kappa partitions (0 = SM count)."""
    _check(load().spmttkrp_plan_repartition(plan.handle, int(kappa), _stream(stream)),
           "spmttkrp_plan_repartition")


def spmttkrp_plan_autotune(plan: Plan, factors, kappas=None, reps: int = 3, stream=None):
    """Time candidate partition counts (default: 1 and 2 per SM) on the given
    factors and leave the plan at the fastest; returns (chosen, ms list)."""
    n = len(kappas) if kappas else 2
    ka = (ctypes.c_int * n)(*[int(k) for k in kappas]) if kappas else None
    ms = (ctypes.c_float * n)()
    chosen = ctypes.c_int()
    _check(load().spmttkrp_plan_autotune(plan.handle, _ptrs(list(factors)), ka,
                                         n if kappas else 0, int(reps), ctypes.byref(chosen),
                                         ms, _stream(stream)),
           "spmttkrp_plan_autotune")
    return int(chosen.value), list(ms)


def spmttkrp_plan_fibre_count(plan: Plan, mode: int) -> int:
    """Fibres (distinct (c_d, c_a) pairs) of a SPM_PLAN_FIBRE plan's mode copy."""
    n = ctypes.c_int64()
    _check(load().spmttkrp_plan_fibre_count(plan.handle, int(mode), ctypes.byref(n)),
           "spmttkrp_plan_fibre_count")
    return int(n.value)


def spmttkrp_plan_destroy(plan: Plan):
    plan.destroy()


def spmttkrp_run(plan: Plan, mode: int, factors, out, stream=None):
    """factors: N CUDA tensors (float32 or bfloat16 per the plan), I_w x R
    row-major (factors[mode] may be None); out: float32 CUDA [I_mode, R]."""
    _check(load().spmttkrp_run(plan.handle, int(mode), _ptrs(list(factors)),
                               ctypes.c_void_p(out.data_ptr()), _stream(stream)),
           "spmttkrp_run")
    return out


def spmttkrp_run_all_host(plan: Plan, host_factors, host_outs, stream=None):
    """MTTKRP along every mode from host (CPU) tensors into host tensors;
    launch-only (synchronise the stream before reading host_outs)."""
    _check(load().spmttkrp_run_all_host(plan.handle, _ptrs(list(host_factors)),
                                        _ptrs(list(host_outs)), _stream(stream)),
           "spmttkrp_run_all_host")


def cpd_als_step(plan: Plan, factors, lam, fit=None, stream=None):
    """One CP-ALS sweep; factors updated in place, lam float64 CUDA [R],
    fit float64 CUDA [1] or None."""
    _check(load().cpd_als_step(plan.handle, _ptrs(list(factors)),
                               ctypes.c_void_p(lam.data_ptr()),
                               ctypes.c_void_p(fit.data_ptr() if fit is not None else 0),
                               _stream(stream)),
           "cpd_als_step")


def cpd_als_reset(plan: Plan):
    """Forget the plan's cached Grams (after writing the factors oneself)."""
    _check(load().cpd_als_reset(plan.handle), "cpd_als_reset")


def spmttkrp_plan_status(plan: Plan, stream=None) -> int:
    """Synchronises and returns (and clears) the plan's device-side status."""
    return int(load().spmttkrp_plan_status(plan.handle, _stream(stream)))


def spmttkrp_run_noalloc(dims, mode: int, rank: int, records, factors, out, flags: int = 0,
                         stream=None):
    """No-allocation MTTKRP from a caller-held mode copy.  records: int32
    CUDA tensor [nnz, 4*ceil((N+1)/4)] in the documented record layout,
    sorted by the output-mode index; factors/out as for spmttkrp_run."""
    N = len(dims)
    dims_a = (ctypes.c_int64 * N)(*[int(d) for d in dims])
    nnz = int(records.shape[0]) if records is not None else 0
    _check(load().spmttkrp_run_noalloc(N, dims_a, nnz, int(mode), int(rank),
                                       ctypes.c_void_p(records.data_ptr() if nnz else 0),
                                       _ptrs(list(factors)), int(flags) & 0xFFFFFFFF,
                                       ctypes.c_void_p(out.data_ptr()), _stream(stream)),
           "spmttkrp_run_noalloc")
    return out


#: largest mode count of the C ABI (factor pointer stride of spm_batch_create)
SPM_MAX_MODES = 7


class Batch:
    """Owns an spm_batch_t: CP-ALS over many tensors, one launch per step for
    all of them.  Keeps references to the plans and buffers it was made from."""

    def __init__(self, handle, plans, factors, lambdas, fits):
        self.handle = handle
        self.plans = list(plans)
        self.factors = [list(f) for f in factors]
        self.lambdas = lambdas
        self.fits = fits
        offs = [0]
        for p in self.plans:
            offs.append(offs[-1] + p.rank)
        self.lambda_offsets = offs

    def lam(self, t: int):
        """Tensor t's weights (a view of the batch's lambda buffer)."""
        return self.lambdas[self.lambda_offsets[t]:self.lambda_offsets[t + 1]]

    def destroy(self):
        if self.handle:
            load().spm_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def spm_batch_create(plans, factors, lambdas, fits, tol: float = 0.0, max_sweeps: int = 1,
                     stream=None) -> Batch:
    """plans: list of Plan; factors: per tensor the list of its N CUDA factor
    tensors (updated in place); lambdas: float64 CUDA [sum of ranks];
    fits: float64 CUDA [len(plans)]."""
    n = len(plans)
    hp = (ctypes.c_void_p * n)(*[p.handle for p in plans])
    fp = (ctypes.c_void_p * (n * SPM_MAX_MODES))()
    for t, fs in enumerate(factors):
        for w, f in enumerate(fs):
            fp[t * SPM_MAX_MODES + w] = f.data_ptr()
    h = ctypes.c_void_p()
    _check(load().spm_batch_create(ctypes.byref(h), n, hp, fp,
                                   ctypes.c_void_p(lambdas.data_ptr()),
                                   ctypes.c_void_p(fits.data_ptr()), float(tol),
                                   int(max_sweeps), _stream(stream)),
           "spm_batch_create")
    return Batch(h, plans, factors, lambdas, fits)


def spm_batch_sweep(batch: Batch, stream=None):
    """One CP-ALS sweep of every still-active tensor (launches only)."""
    _check(load().spm_batch_sweep(batch.handle, _stream(stream)), "spm_batch_sweep")


def spm_batch_status(batch: Batch, stream=None):
    """Synchronises; returns (active, sweeps) as lists of ints."""
    n = len(batch.plans)
    act = (ctypes.c_int * n)()
    sw = (ctypes.c_int * n)()
    _check(load().spm_batch_status(batch.handle, act, sw, _stream(stream)), "spm_batch_status")
    return list(act), list(sw)


def spm_batch_destroy(batch: Batch):
    batch.destroy()


def spm_batch_autotune(plans, factors, candidates=(0, 1 << 12, 1 << 14, 1 << 16, 1 << 18),
                       reps: int = 3, stream=None):
    """Pick the nonzeros per partition for a batch; returns (chosen, ms per
    candidate).  The plans are left partitioned for the chosen value."""
    n = len(plans)
    hp = (ctypes.c_void_p * n)(*[p.handle for p in plans])
    fp = (ctypes.c_void_p * (n * SPM_MAX_MODES))()
    for t, fs in enumerate(factors):
        for w, f in enumerate(fs):
            fp[t * SPM_MAX_MODES + w] = f.data_ptr()
    cand = (ctypes.c_int64 * len(candidates))(*[int(c) for c in candidates])
    ms = (ctypes.c_float * len(candidates))()
    chosen = ctypes.c_int64()
    _check(load().spm_batch_autotune(n, hp, fp, cand, len(candidates), int(reps),
                                     ctypes.byref(chosen), ms, _stream(stream)),
           "spm_batch_autotune")
    return int(chosen.value), list(ms)


def spmttkrp_plan_bytes_estimate(dims, nnz: int, rank: int, flags: int = 0):
    """(resident, transient) device bytes of a plan of this shape (host only)."""
    N = len(dims)
    dims_a = (ctypes.c_int64 * N)(*[int(d) for d in dims])
    res, tr = ctypes.c_size_t(), ctypes.c_size_t()
    _check(load().spmttkrp_plan_bytes_estimate(N, dims_a, int(nnz), int(rank),
                                               int(flags) & 0xFFFFFFFF, ctypes.byref(res),
                                               ctypes.byref(tr)),
           "spmttkrp_plan_bytes_estimate")
    return int(res.value), int(tr.value)


SPM_JOB_QUEUED, SPM_JOB_RUNNING, SPM_JOB_DONE, SPM_JOB_FAILED = 0, 1, 2, 3


class JobDesc(ctypes.Structure):
    _fields_ = [("nmodes", ctypes.c_int), ("dims", ctypes.c_void_p), ("nnz", ctypes.c_int64),
                ("idx", ctypes.c_void_p), ("vals", ctypes.c_void_p), ("rank", ctypes.c_int),
                ("init", ctypes.c_void_p), ("tol", ctypes.c_double),
                ("max_sweeps", ctypes.c_int)]


class JobInfo(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int), ("status", ctypes.c_int), ("sweeps", ctypes.c_int),
                ("fit", ctypes.c_double), ("bytes", ctypes.c_size_t),
                ("est_bytes", ctypes.c_size_t), ("queued_ms", ctypes.c_double),
                ("total_ms", ctypes.c_double)]


class Server:
    """Owns an spm_server_t (continuous batching of CP-ALS jobs).  Keeps the
    submitted input tensors alive until their jobs are admitted."""

    def __init__(self, budget_bytes: int, max_active: int = 64, flags: int = 0,
                 nnz_per_partition: int = 1 << 17):
        h = ctypes.c_void_p()
        _check(load().spm_server_create(ctypes.byref(h), int(budget_bytes), int(max_active),
                                        int(flags), int(nnz_per_partition)),
               "spm_server_create")
        self.handle = h
        self.flags = int(flags)
        self._inputs = {}
        self.ranks = {}
        self.shapes = {}

    def submit(self, dims, idx, vals, rank: int, init, tol: float = 1e-4,
               max_sweeps: int = 50, resume=None) -> int:
        """idx: N int32 CUDA tensors, vals float32 CUDA, init: N float32 CUDA
        [I_w, R].  The producing stream must be synchronised first.
        resume = (sweeps_done, prev_fit) from a snapshot continues that job
        (init then holds the snapshot's factors as FP32)."""
        N = len(dims)
        dims_a = (ctypes.c_int64 * N)(*[int(d) for d in dims])
        idx_a = (ctypes.c_void_p * N)(*[c.data_ptr() for c in idx])
        init_a = (ctypes.c_void_p * N)(*[f.data_ptr() for f in init])
        nnz = int(vals.numel())
        d = JobDesc(N, ctypes.cast(dims_a, ctypes.c_void_p).value, nnz,
                    ctypes.cast(idx_a, ctypes.c_void_p).value if nnz else None,
                    vals.data_ptr() if nnz else None, int(rank),
                    ctypes.cast(init_a, ctypes.c_void_p).value, float(tol), int(max_sweeps))
        job = ctypes.c_int64()
        if resume is None:
            _check(load().spm_server_submit(self.handle, ctypes.byref(d), ctypes.byref(job)),
                   "spm_server_submit")
        else:
            _check(load().spm_server_resume(self.handle, ctypes.byref(d), int(resume[0]),
                                            float(resume[1]), ctypes.byref(job)),
                   "spm_server_resume")
        j = int(job.value)
        self._inputs[j] = (idx, vals, init)
        self.ranks[j] = int(rank)
        self.shapes[j] = tuple(int(x) for x in dims)
        return j

    def step(self):
        """One step; returns (running, queued)."""
        r, q = ctypes.c_int(), ctypes.c_int()
        _check(load().spm_server_step(self.handle, ctypes.byref(r), ctypes.byref(q)),
               "spm_server_step")
        for j in list(self._inputs):
            if self.info(j).state != SPM_JOB_QUEUED:
                del self._inputs[j]
        return int(r.value), int(q.value)

    def info(self, job: int) -> JobInfo:
        i = JobInfo()
        _check(load().spm_server_job(self.handle, int(job), ctypes.byref(i)), "spm_server_job")
        return i

    def result(self, job: int, stream=None):
        """(factors, lambda) of a finished job as new CUDA tensors; releases it."""
        import torch
        dt = torch.bfloat16 if self.flags & SPM_FACTOR_BF16 else torch.float32
        R = self.ranks[job]
        fac = [torch.empty(n, R, dtype=dt, device="cuda") for n in self.shapes[job]]
        lam = torch.empty(R, dtype=torch.float64, device="cuda")
        _check(load().spm_server_result(self.handle, int(job), _ptrs(fac),
                                        ctypes.c_void_p(lam.data_ptr()), _stream(stream)),
               "spm_server_result")
        return fac, lam

    def snapshot(self, job: int, stream=None):
        """(factors, lambda, sweeps_done, prev_fit) of a running job, between steps."""
        import torch
        dt = torch.bfloat16 if self.flags & SPM_FACTOR_BF16 else torch.float32
        R = self.ranks[job]
        fac = [torch.empty(n, R, dtype=dt, device="cuda") for n in self.shapes[job]]
        lam = torch.empty(R, dtype=torch.float64, device="cuda")
        sw, pf = ctypes.c_int(), ctypes.c_double()
        _check(load().spm_server_snapshot(self.handle, int(job), _ptrs(fac),
                                          ctypes.c_void_p(lam.data_ptr()), ctypes.byref(sw),
                                          ctypes.byref(pf), _stream(stream)),
               "spm_server_snapshot")
        return fac, lam, int(sw.value), float(pf.value)

    def usage(self):
        u, b = ctypes.c_size_t(), ctypes.c_size_t()
        _check(load().spm_server_usage(self.handle, ctypes.byref(u), ctypes.byref(b)),
               "spm_server_usage")
        return int(u.value), int(b.value)

    def destroy(self):
        if self.handle:
            load().spm_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def spm_selftest_wait_timeout(limit: int = 4096, stream=None) -> int:
    """Status of the bounded-wait self-test (SPM_ERR_TIMEOUT expected)."""
    return int(load().spm_selftest_wait_timeout(int(limit), _stream(stream)))


def spm_selftest_mttkrp_timeout(plan, mode: int, factors, out, stream=None) -> int:
    """Status of the plan's MTTKRP run with record-copy waits that give up at
    once (SPM_ERR_TIMEOUT expected)."""
    return int(load().spm_selftest_mttkrp_timeout(plan.handle, int(mode), _ptrs(list(factors)),
                                                  ctypes.c_void_p(out.data_ptr()),
                                                  _stream(stream)))


def spm_selftest_tc_rowpass(M, V, stream=None):
    """The CP-ALS row passes of one mode on caller data: M (I x R float32
    CUDA), V (R x R float64 CUDA, SPD).  Returns (Z, Y, G, lam): Z = M V^-1,
    Y = Z / lam (float32), G = Y^T Y (float64; R = 16, 32 only, else zeros),
    lam = column 2-norms of Z (float64)."""
    import torch
    I, R = M.shape
    Z = torch.empty_like(M)
    Y = torch.empty_like(M)
    G = torch.zeros(R, R, dtype=torch.float64, device=M.device)
    lam = torch.empty(R, dtype=torch.float64, device=M.device)
    _check(load().spm_selftest_tc_rowpass(int(R), int(I), ctypes.c_void_p(M.data_ptr()),
                                          ctypes.c_void_p(V.data_ptr()),
                                          ctypes.c_void_p(Z.data_ptr()),
                                          ctypes.c_void_p(Y.data_ptr()),
                                          ctypes.c_void_p(G.data_ptr()),
                                          ctypes.c_void_p(lam.data_ptr()), _stream(stream)),
           "spm_selftest_tc_rowpass")
    return Z, Y, G, lam


def spmttkrp_noalloc_status(stream=None) -> int:
    """Device-side outcome of the latest spmttkrp_run_noalloc call (a status
    code; synchronises the stream)."""
    return int(load().spmttkrp_noalloc_status(_stream(stream)))


def spm_inject_alloc_failure(k: int):
    """Make the k-th plan allocation from now fail with SPM_ERR_OOM (k < 0: off)."""
    load().spm_inject_alloc_failure(int(k))


# Same-named functions for the serving entry points (the Server methods do the
# marshalling).
def spm_server_create(budget_bytes: int, max_active: int = 64, flags: int = 0,
                      nnz_per_partition: int = 1 << 17) -> Server:
    return Server(budget_bytes, max_active, flags, nnz_per_partition)


def spm_server_submit(server: Server, dims, idx, vals, rank: int, init, tol: float = 1e-4,
                      max_sweeps: int = 50) -> int:
    return server.submit(dims, idx, vals, rank, init, tol, max_sweeps)


def spm_server_resume(server: Server, dims, idx, vals, rank: int, init, sweeps_done: int,
                      prev_fit: float, tol: float = 1e-4, max_sweeps: int = 50) -> int:
    return server.submit(dims, idx, vals, rank, init, tol, max_sweeps,
                         resume=(sweeps_done, prev_fit))


def spm_server_step(server: Server):
    return server.step()


def spm_server_job(server: Server, job: int) -> JobInfo:
    return server.info(job)


def spm_server_result(server: Server, job: int, stream=None):
    return server.result(job, stream)


def spm_server_snapshot(server: Server, job: int, stream=None):
    return server.snapshot(job, stream)


def spm_server_usage(server: Server):
    return server.usage()


def spm_server_destroy(server: Server):
    server.destroy()
