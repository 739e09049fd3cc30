"""Parity at the full workload sizes, in the launch configuration bench.py
times (default plan: cost-balanced work units, two partitions per SM).

* scale: 1,000,000 x 500,000 x 200,000, 50M nonzeros, Zipf(1.2), R = 32 FP32.
* precision: 20,000 x 20,000 x 5,000 x 24, 100M nonzeros, Zipf(1.0) x3 +
  uniform, lognormal values, R = 64, BF16 and FP32 factors.

The oracle cannot form full outputs of this size quickly, so it computes
sampled output rows one by one (the heaviest rows, the rows at partition and
work-unit boundaries, random non-empty rows; empty rows must be exactly 0).
The copy order is checked at full size by properties that determine it
uniquely (a permutation whose (key, position) sequence strictly increases),
and the partition against the oracle's formula applied to the sorted
output-mode indices computed on the host.
"""
import numpy as np
import pytest

import oracle
import synth
from parity_util import check_rows_elementwise

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2503_18198_gb300 as spm  # noqa: E402

TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    spm.load(build_if_missing=True)


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def check_order(perm, idx_h, d):
    """perm is a permutation and the (c_d, other modes ascending, position)
    keys strictly increase along it -- which fixes it uniquely."""
    n = perm.size
    seen = np.zeros(n, dtype=bool)
    seen[perm] = True
    assert seen.all()
    keys = [idx_h[d][perm]] + [idx_h[w][perm] for w in range(len(idx_h)) if w != d] + [perm]
    undecided = np.ones(n - 1, dtype=bool)  # pairs (k, k+1) equal so far
    for key in keys:
        a, b = key[:-1], key[1:]
        assert not np.any(undecided & (a > b))
        undecided &= (a == b)
    assert not undecided.any()


def sample_rows(idx_h, d, dim, units, rng):
    deg = np.bincount(idx_h[d], minlength=dim)
    heavy = np.argsort(-deg, kind="stable")[:5]
    rows_sorted = np.sort(idx_h[d])
    bnd = np.unique(np.concatenate([rows_sorted[np.minimum(units[:-1], rows_sorted.size - 1)],
                                    rows_sorted[np.maximum(units[1:] - 1, 0)]]))
    bnd = rng.choice(bnd, size=min(200, bnd.size), replace=False)
    nonempty = np.nonzero(deg)[0]
    rnd = rng.choice(nonempty, size=min(200, nonempty.size), replace=False)
    empty = np.nonzero(deg == 0)[0]
    empty = rng.choice(empty, size=min(50, empty.size), replace=False) if empty.size else empty
    rows = np.unique(np.concatenate([heavy, bnd, rnd])).astype(np.int32)
    return rows, empty.astype(np.int64), rows_sorted


def run_fullsize(name, dtype, flags, check_structure):
    dims, idx, vals, R, Y = synth.preset_torch(name, device="cuda")
    N = len(dims)
    plan = spm.spmttkrp_plan(dims, idx, vals, R, flags)
    fac = [y.to(dtype).contiguous() for y in Y]
    idx_h = [c.cpu().numpy() for c in idx]
    vals_h = vals.cpu().numpy()
    fac_h = [f.float().cpu().numpy() for f in fac]   # the factors the GPU used
    kappa = spm.binding.default_kappa()
    U = spm.SPM_UNITS_PER_PARTITION(R)
    rng = np.random.default_rng(7)
    for d in range(N):
        out = torch.empty(dims[d], R, device="cuda")
        spm.spmttkrp_run(plan, d, fac, out)
        units = torch.empty(kappa * U + 1, dtype=torch.int64, device="cuda")
        spm.spmttkrp_plan_work_units(plan, d, units)
        units = units.cpu().numpy()
        rows, empty, rows_sorted = sample_rows(idx_h, d, dims[d], units, rng)
        if check_structure:
            perm = torch.empty(plan.nnz, dtype=torch.int64, device="cuda")
            spm.spmttkrp_plan_permutation(plan, d, perm)
            check_order(perm.cpu().numpy(), idx_h, d)
            ref_units = oracle.partition_balanced_rows(rows_sorted, kappa * U, spm.SPM_ROW_COST)
            assert np.array_equal(units, ref_units)
        got = out.cpu().numpy()
        ref = check_rows_elementwise(got[rows], dims, idx_h, vals_h, fac_h, d, rows,
                                     what=f"{name} mode {d}")
        assert rel(got[rows], ref) < TOL, f"{name} mode {d}"
        heavy = rows[np.argmax(np.abs(ref).sum(axis=1))]
        assert rel(got[heavy], ref[np.searchsorted(rows, heavy)]) < TOL
        if empty.size:
            assert np.all(got[empty] == 0.0)
    plan.destroy()
    return dims, idx_h, vals_h, Y


def test_scale_workload_fp32():
    run_fullsize("scale", torch.float32, 0, check_structure=True)


@pytest.mark.parametrize("dtype,flags", [(torch.float32, 0),
                                         (torch.bfloat16, spm.SPM_FACTOR_BF16)])
def test_precision_workload(dtype, flags):
    run_fullsize("precision", dtype, flags, check_structure=(dtype == torch.float32))
