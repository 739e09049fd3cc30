"""Memory-lean plans (SPM_PLAN_LEAN): one record copy (mode 0) plus, for
every other mode, the mode's order as positions into that copy.

The lean MTTKRP visits the nonzeros of a mode in the same order and does the
same arithmetic as the full plan's, so every output, permutation, partition
and CP-ALS sweep is compared with the full plan bitwise; the full plan is
itself checked against the FP64 oracle elsewhere (and here once more).
"""
import numpy as np
import pytest

import oracle
import synth
from parity_util import check_mode_elementwise

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2503_18198_gb300 as spm  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    spm.load(build_if_missing=True)


CASES = [
    # dims, nnz, R, alphas, kappa (0 = default)
    ((300, 200, 100), 20000, 16, (1.2, 1.2, 1.2), 0),
    ((1000, 50, 70), 60000, 32, (1.1, None, 1.1), 7),
    ((64, 48, 32, 6), 5000, 64, (None, None, None, None), 3),
    ((25, 25, 25, 25), 3000, 8, (1.0, 1.0, None, None), 0),
    ((400, 90, 2, 30, 11), 40000, 32, (1.1, 1.1, None, None, None), 40),
]


def build(dims, nnz, R, alphas, seed, flags):
    dims, idx, vals = synth.coo_distinct(dims, nnz, alphas, seed=seed)
    didx = [torch.as_tensor(c).cuda() for c in idx]
    dvals = torch.as_tensor(vals).cuda()
    return dims, idx, vals, spm.spmttkrp_plan(dims, didx, dvals, R, flags)


def copies(plan, d, kappa):
    n = plan.nnz
    perm = torch.empty(n, dtype=torch.int64, device="cuda")
    spm.spmttkrp_plan_permutation(plan, d, perm)
    off = torch.empty(kappa + 1, dtype=torch.int64, device="cuda")
    spm.spmttkrp_plan_partition(plan, d, off)
    U = spm.SPM_UNITS_PER_PARTITION(plan.rank)
    units = torch.empty(kappa * U + 1, dtype=torch.int64, device="cuda")
    spm.spmttkrp_plan_work_units(plan, d, units)
    return perm, off, units


def bits(t):
    return t.view(torch.int16) if t.dtype == torch.bfloat16 else t


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("dtype,fflag", [(torch.float32, spm.SPM_FACTOR_FP32),
                                         (torch.bfloat16, spm.SPM_FACTOR_BF16)])
def test_lean_plan_equals_full_plan_bitwise(case, dtype, fflag):
    dims, nnz, R, alphas, k = CASES[case]
    flags = fflag | spm.SPM_KAPPA(k)
    dims, idx, vals, full = build(dims, nnz, R, alphas, 60 + case, flags)
    _, _, _, lean = build(dims, nnz, R, alphas, 60 + case, flags | spm.SPM_PLAN_LEAN)
    N = len(dims)
    kappa = k or spm.binding.default_kappa()
    Y = [torch.as_tensor(f).to(dtype).cuda().contiguous()
         for f in synth.factors(dims, R, seed=case)]
    for d in range(N):
        for a, b in zip(copies(full, d, kappa), copies(lean, d, kappa)):
            assert torch.equal(a, b), f"mode {d} structure"
        of = torch.empty(dims[d], R, device="cuda")
        ol = torch.full((dims[d], R), float("nan"), device="cuda")
        spm.spmttkrp_run(full, d, Y, of)
        spm.spmttkrp_run(lean, d, Y, ol)
        assert torch.equal(of, ol), f"mode {d} output"
        if case == 0 and dtype == torch.float32:
            got = ol.double().cpu().numpy()
            ref = check_mode_elementwise(got, dims, idx, vals,
                                         [y.double().cpu().numpy() for y in Y], d)
            assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-5
    # CP-ALS on both plans from the same factors
    fa = [y.clone() for y in Y]
    fb = [y.clone() for y in Y]
    la = torch.zeros(R, dtype=torch.float64, device="cuda")
    lb = torch.zeros(R, dtype=torch.float64, device="cuda")
    ta = torch.zeros(1, dtype=torch.float64, device="cuda")
    tb = torch.zeros(1, dtype=torch.float64, device="cuda")
    for _ in range(2):
        spm.cpd_als_step(full, fa, la, ta)
        spm.cpd_als_step(lean, fb, lb, tb)
    for a, b in zip(fa, fb):
        assert torch.equal(bits(a), bits(b))
    assert torch.equal(la, lb) and torch.equal(ta, tb)
    assert spm.spmttkrp_plan_status(full) == 0 and spm.spmttkrp_plan_status(lean) == 0
    # memory: one record copy instead of N
    bf, bl = spm.spmttkrp_plan_bytes(full), spm.spmttkrp_plan_bytes(lean)
    est, _ = spm.spmttkrp_plan_bytes_estimate(dims, nnz, R, flags | spm.SPM_PLAN_LEAN)
    assert bl == est
    assert bl < bf


def test_lean_repartition_autotune_and_restrictions():
    dims, nnz, R, alphas, _ = CASES[1]
    dims, idx, vals, full = build(dims, nnz, R, alphas, 7, 0)
    _, _, _, lean = build(dims, nnz, R, alphas, 7, spm.SPM_PLAN_LEAN)
    Y = [torch.as_tensor(f).cuda() for f in synth.factors(dims, R, seed=7)]
    for k in (5, 300):
        spm.spmttkrp_plan_repartition(full, k)
        spm.spmttkrp_plan_repartition(lean, k)
        for d in range(3):
            for a, b in zip(copies(full, d, k), copies(lean, d, k)):
                assert torch.equal(a, b)
            of = torch.empty(dims[d], R, device="cuda")
            ol = torch.empty(dims[d], R, device="cuda")
            spm.spmttkrp_run(full, d, Y, of)
            spm.spmttkrp_run(lean, d, Y, ol)
            assert torch.equal(of, ol)
    chosen, _ = spm.spmttkrp_plan_autotune(lean, Y)
    assert chosen in (spm.spm_device_sm_count(), 2 * spm.spm_device_sm_count())
    didx = [torch.as_tensor(c).cuda() for c in idx]
    dvals = torch.as_tensor(vals).cuda()
    for pol in (spm.SPM_POLICY_SCHEME1, spm.SPM_POLICY_ADAPTIVE):
        with pytest.raises(spm.SpmError) as e:
            spm.spmttkrp_plan(dims, didx, dvals, R, pol | spm.SPM_PLAN_LEAN)
        assert e.value.status == 7
    lam = torch.zeros(R, dtype=torch.float64, device="cuda")
    fits = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(spm.SpmError) as e:
        spm.spm_batch_create([lean], [Y], lam, fits)
    assert e.value.status == 7


@pytest.mark.parametrize("nnz,dup", [(0, False), (1, False), (3000, True)])
def test_lean_edge_cases(nnz, dup):
    """Empty and one-nonzero tensors, and repeated coordinates (summed)."""
    dims = (40, 30, 20)
    if nnz == 0:
        idx = [np.zeros(0, np.int32) for _ in dims]
        vals = np.zeros(0, np.float32)
    else:
        _, idx, vals = synth.coo_random(dims, nnz, seed=11, duplicates=dup)
    didx = [torch.as_tensor(c).cuda() for c in idx]
    dvals = torch.as_tensor(vals).cuda()
    full = spm.spmttkrp_plan(dims, didx, dvals, 16)
    lean = spm.spmttkrp_plan(dims, didx, dvals, 16, spm.SPM_PLAN_LEAN)
    Y = [torch.as_tensor(f).cuda() for f in synth.factors(dims, 16, seed=11)]
    for d in range(3):
        of = torch.full((dims[d], 16), float("nan"), device="cuda")
        ol = torch.full((dims[d], 16), float("nan"), device="cuda")
        spm.spmttkrp_run(full, d, Y, of)
        spm.spmttkrp_run(lean, d, Y, ol)
        assert torch.equal(of, ol)
        if nnz:
            got = ol.double().cpu().numpy()
            ref = check_mode_elementwise(got, dims, idx, vals,
                                         [y.double().cpu().numpy() for y in Y], d)
            assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-5
        else:
            assert torch.count_nonzero(ol) == 0
