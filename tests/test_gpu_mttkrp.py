"""GPU parity of the mode copies, partitions and MTTKRP against the oracle.

Every case calls the CUDA library through the C ABI (ctypes binding) and
compares with the FP64 oracle on the same seeded inputs:
  * permutations and partition offsets bit-exactly;
  * FP32 MTTKRP within 1e-5 relative Frobenius error per mode;
  * BF16 factors: against the oracle on the same BF16-rounded factors (the
    accumulation error, same 1e-5 bound) and against the FP32 factors (the
    total error, bounded by the BF16 rounding of the inputs).
"""
import numpy as np
import pytest

import oracle
import synth
from parity_util import check_mode_elementwise

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2503_18198_gb300 as spm  # noqa: E402

TOL = 1e-5  # relative Frobenius error per mode (FP32 accumulation)


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def to_dev(dims, idx, vals):
    return ([torch.as_tensor(c, dtype=torch.int32).cuda() for c in idx],
            torch.as_tensor(np.asarray(vals, np.float32)).cuda())


def run_all_modes(dims, idx, vals, factors, flags=0, dtype=torch.float32):
    didx, dvals = to_dev(dims, idx, vals)
    R = factors[0].shape[1]
    plan = spm.spmttkrp_plan(dims, didx, dvals, R, flags)
    dfac = [torch.as_tensor(f).to(dtype).cuda().contiguous() for f in factors]
    outs = []
    for d in range(len(dims)):
        out = torch.full((dims[d], R), float("nan"), dtype=torch.float32, device="cuda")
        spm.spmttkrp_run(plan, d, dfac, out)
        outs.append(out)
    torch.cuda.synchronize()
    return plan, [o.cpu().numpy() for o in outs], dfac


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    spm.load(build_if_missing=True)


def check_copies(plan, idx, kappa=None, policy="balanced"):
    """Permutation, partition offsets and work-unit offsets of every mode copy
    against the oracle, bit-exactly."""
    dims = plan.dims
    U = spm.SPM_UNITS_PER_PARTITION(plan.rank)
    for d in range(len(dims)):
        perm = torch.empty(plan.nnz, dtype=torch.int64, device="cuda")
        spm.spmttkrp_plan_permutation(plan, d, perm)
        ref = oracle.mode_permutation(idx, d)
        assert np.array_equal(perm.cpu().numpy(), ref), f"mode {d} permutation"
        k = kappa or spm.binding.default_kappa()
        off = torch.empty(k + 1, dtype=torch.int64, device="cuda")
        assert spm.spmttkrp_plan_partition(plan, d, off) == k
        units = torch.empty(k * U + 1, dtype=torch.int64, device="cuda")
        spm.spmttkrp_plan_work_units(plan, d, units)
        if policy == "balanced":
            ref_units = oracle.partition_balanced(idx, d, k * U, spm.SPM_ROW_COST, perm=ref)
            ref_off = ref_units[::U]
        else:
            ref_off = oracle.partition_equal(plan.nnz, k)
            ref_units = oracle.units_from_partitions(ref_off, U)
        assert np.array_equal(off.cpu().numpy(), ref_off), f"mode {d} partition"
        assert np.array_equal(units.cpu().numpy(), ref_units), f"mode {d} work units"


def test_plain_workload_all_modes():
    """64x48x32, 4096 distinct uniform nonzeros, R = 16 (the plain workload)."""
    dims, idx, vals, R, Y = synth.preset("plain")
    plan, outs, _ = run_all_modes(dims, idx, vals, Y)
    check_copies(plan, idx)
    for d in range(3):
        ref = check_mode_elementwise(outs[d], dims, idx, vals, Y, d)
        assert rel(outs[d], ref) < TOL


@pytest.mark.parametrize("dims,R,nnz,kappa", [
    ((37, 29, 23), 32, 3000, 7),      # several partitions, ragged tail
    ((50, 40, 30), 16, 5000, 3),
    ((9, 8, 7, 6), 8, 1500, 5),       # 4 modes
    ((6, 5, 4, 5, 3), 16, 800, 4),    # 5 modes (two 16-byte record words)
    ((300, 2), 64, 500, 11),          # 2 modes
    ((20, 30, 40), 1, 2000, 9),       # rank 1 (scalar path)
    ((20, 30, 40), 24, 2000, 9),      # rank not a power of two
    ((20, 30, 40), 100, 1000, 6),     # odd rank, scalar path
    ((20, 30, 40), 128, 1000, 6),
    ((20, 30, 40), 256, 600, 5),      # maximum rank
    ((1000, 12, 11), 32, 4000, 152),  # empty rows in mode 0
    ((3, 1000, 5), 32, 6000, 152),    # tiny output mode: every partition on 3 rows
])
def test_random_shapes(dims, R, nnz, kappa):
    g = np.random.default_rng(sum(dims) + R + nnz)
    idx = [g.integers(0, n, nnz).astype(np.int32) for n in dims]   # duplicates too
    vals = g.random(nnz).astype(np.float32)
    Y = [g.standard_normal((n, R)).astype(np.float32) for n in dims]
    plan, outs, _ = run_all_modes(dims, idx, vals, Y, spm.SPM_KAPPA(kappa))
    check_copies(plan, idx, kappa)
    for d in range(len(dims)):
        ref = check_mode_elementwise(outs[d], dims, idx, vals, Y, d)
        assert rel(outs[d], ref) < TOL, f"mode {d}"


def test_heavy_row_dominated():
    """Most nonzeros on one output row of every mode (a Zipf head): the row
    spans many warps and partitions and is combined by the fix-up."""
    g = np.random.default_rng(7)
    dims, R, nnz = (400, 300, 200), 32, 60000
    idx = [np.where(g.random(nnz) < 0.6, 0, g.integers(0, n, nnz)).astype(np.int32)
           for n in dims]
    vals = g.random(nnz).astype(np.float32)
    Y = [g.standard_normal((n, R)).astype(np.float32) for n in dims]
    for kappa in (152, 13):
        plan, outs, _ = run_all_modes(dims, idx, vals, Y, spm.SPM_KAPPA(kappa))
        for d in range(3):
            ref = check_mode_elementwise(outs[d], dims, idx, vals, Y, d)
            assert rel(outs[d], ref) < TOL
            assert rel(outs[d][0], ref[0]) < TOL


def test_zipf_scale_recipe_small():
    dims, idx, vals = synth.coo_distinct((20000, 10000, 4000), 200000, (1.2, 1.2, 1.2), seed=5)
    Y = synth.factors(dims, 32, seed=5)
    plan, outs, _ = run_all_modes(dims, idx, vals, Y)
    check_copies(plan, idx)
    for d in range(3):
        ref = check_mode_elementwise(outs[d], dims, idx, vals, Y, d)
        assert rel(outs[d], ref) < TOL


@pytest.mark.parametrize("R", [8, 16, 32, 64, 12])
def test_bf16_factors(R):
    dims, idx, vals = synth.coo_distinct((500, 400, 300, 24), 20000, (1.0, 1.0, 1.0, None),
                                         seed=R, values="lognormal")
    Y = synth.factors(dims, R, seed=R)
    plan, outs, dfac = run_all_modes(dims, idx, vals, Y, spm.SPM_FACTOR_BF16,
                                     dtype=torch.bfloat16)
    Yb = [f.float().cpu().numpy() for f in dfac]
    for d in range(4):
        ref_same = check_mode_elementwise(outs[d], dims, idx, vals, Yb, d)
        ref_fp32 = oracle.mttkrp(dims, idx, vals, Y, d)
        assert rel(outs[d], ref_same) < TOL          # accumulation error
        assert rel(outs[d], ref_fp32) < 2e-2         # includes BF16 input rounding


@pytest.mark.parametrize("dims,R,nnz", [
    ((3000, 200, 100), 8, 20000),       # 3 modes, R <= 32: 8-byte BF16 lanes
    ((3000, 200, 100), 16, 20000),
    ((3001, 203, 97), 24, 20000),       # rank not a power of two
    ((3000, 200, 100), 32, 20000),
    ((3000, 200, 100), 64, 20000),      # 16-byte lanes
    ((400, 30, 3, 20, 17), 16, 6000),   # 5 modes
    ((400, 30, 3, 20, 17), 32, 6000),
])
def test_bf16_factors_three_and_five_modes(dims, R, nnz):
    """BF16 factors widen straight into FP32 pairs; element-wise parity for
    every mode against the oracle on the same BF16 values, with Zipf heads,
    duplicates removed, ragged tiles and empty rows."""
    alphas = (1.1, 1.1) + (None,) * (len(dims) - 2)
    dims, idx, vals = synth.coo_distinct(dims, nnz, alphas, seed=R + len(dims))
    assert len(np.unique(idx[0])) < dims[0]  # mode 0 has empty rows
    Y = synth.factors(dims, R, seed=R + len(dims))
    plan, outs, dfac = run_all_modes(dims, idx, vals, Y, spm.SPM_FACTOR_BF16,
                                     dtype=torch.bfloat16)
    Yb = [f.float().cpu().numpy() for f in dfac]
    for d in range(len(dims)):
        ref = check_mode_elementwise(outs[d], dims, idx, vals, Yb, d)
        assert rel(outs[d], ref) < TOL, f"mode {d}"
        assert rel(outs[d], oracle.mttkrp(dims, idx, vals, Y, d)) < 2e-2


def test_scheme2_policy():
    g = np.random.default_rng(11)
    dims, R, nnz, kappa = (70, 60, 50), 32, 9000, 17
    idx = [g.integers(0, n, nnz).astype(np.int32) for n in dims]
    vals = g.random(nnz).astype(np.float32)
    Y = [g.standard_normal((n, R)).astype(np.float32) for n in dims]
    plan, outs, _ = run_all_modes(dims, idx, vals, Y,
                                  spm.SPM_POLICY_SCHEME2 | spm.SPM_KAPPA(kappa))
    check_copies(plan, idx, kappa, policy="scheme2")
    for d in range(3):
        assert spm.spmttkrp_plan_scheme(plan, d) == 2
        ref = check_mode_elementwise(outs[d], dims, idx, vals, Y, d)
        assert rel(outs[d], ref) < TOL


@pytest.mark.parametrize("policy", ["scheme1", "adaptive"])
def test_scheme1_and_adaptive(policy):
    g = np.random.default_rng(3)
    dims, R, nnz, kappa = (60, 9, 45), 16, 4000, 10   # mode 1 has I_d < kappa
    idx = [g.integers(0, n, nnz).astype(np.int32) for n in dims]
    vals = g.random(nnz).astype(np.float32)
    Y = [g.standard_normal((n, R)).astype(np.float32) for n in dims]
    flag = spm.SPM_POLICY_SCHEME1 if policy == "scheme1" else spm.SPM_POLICY_ADAPTIVE
    plan, outs, _ = run_all_modes(dims, idx, vals, Y, flag | spm.SPM_KAPPA(kappa))
    for d in range(3):
        scheme = spm.spmttkrp_plan_scheme(plan, d)
        want = 1 if policy == "scheme1" else oracle.adaptive_policy(dims[d], kappa)
        assert scheme == want
        perm = torch.empty(nnz, dtype=torch.int64, device="cuda")
        spm.spmttkrp_plan_permutation(plan, d, perm)
        off = torch.empty(kappa + 1, dtype=torch.int64, device="cuda")
        spm.spmttkrp_plan_partition(plan, d, off)
        if scheme == 1:
            p1, o1, _ = oracle.partition_scheme1(dims, idx, d, kappa)
        else:
            p1, o1 = oracle.mode_permutation(idx, d), oracle.partition_equal(nnz, kappa)
        assert np.array_equal(perm.cpu().numpy(), p1)
        assert np.array_equal(off.cpu().numpy(), o1)
        U = spm.SPM_UNITS_PER_PARTITION(R)
        units = torch.empty(kappa * U + 1, dtype=torch.int64, device="cuda")
        spm.spmttkrp_plan_work_units(plan, d, units)
        assert np.array_equal(units.cpu().numpy(), oracle.units_from_partitions(o1, U))
        ref = check_mode_elementwise(outs[d], dims, idx, vals, Y, d)
        assert rel(outs[d], ref) < TOL


def test_edge_cases_empty_single_and_repeat():
    dims, R = (5, 4, 3), 8
    Y = synth.factors(dims, R, seed=1)
    # empty tensor: every output row is zero
    plan, outs, _ = run_all_modes(dims, [np.zeros(0, np.int32)] * 3, np.zeros(0, np.float32), Y)
    assert all(np.all(o == 0) for o in outs)
    # one nonzero
    idx = [np.array([4], np.int32), np.array([0], np.int32), np.array([2], np.int32)]
    plan, outs, _ = run_all_modes(dims, idx, np.array([2.0], np.float32), Y)
    for d in range(3):
        ref = check_mode_elementwise(outs[d], dims, idx, [2.0], Y, d)
        assert rel(outs[d], ref) < TOL
    # repeated calls are bitwise identical
    g = np.random.default_rng(0)
    idx = [g.integers(0, n, 3000).astype(np.int32) for n in (80, 70, 60)]
    vals = g.random(3000).astype(np.float32)
    Y = synth.factors((80, 70, 60), 32, seed=3)
    didx, dvals = to_dev((80, 70, 60), idx, vals)
    plan = spm.spmttkrp_plan((80, 70, 60), didx, dvals, 32, spm.SPM_KAPPA(9))
    dfac = [torch.as_tensor(f).cuda() for f in Y]
    a = torch.empty(80, 32, device="cuda")
    b = torch.empty(80, 32, device="cuda")
    spm.spmttkrp_run(plan, 0, dfac, a)
    spm.spmttkrp_run(plan, 0, dfac, b)
    assert torch.equal(a, b)


def test_index_out_of_range_reported():
    idx = [torch.tensor([0, 7], dtype=torch.int32, device="cuda"),
           torch.tensor([1, 1], dtype=torch.int32, device="cuda")]
    vals = torch.ones(2, device="cuda")
    with pytest.raises(spm.SpmError) as e:
        spm.spmttkrp_plan((4, 2), idx, vals, 4)
    assert e.value.status == 2
    idx[0][1] = -1
    with pytest.raises(spm.SpmError):
        spm.spmttkrp_plan((4, 2), idx, vals, 4)


def test_plan_bytes_counts_copies():
    dims, idx, vals, R, Y = synth.preset("plain")
    didx, dvals = to_dev(dims, idx, vals)
    plan = spm.spmttkrp_plan(dims, didx, dvals, R)
    b = spm.spmttkrp_plan_bytes(plan)
    assert b >= 3 * 4096 * (16 + 4)   # three 16-byte record copies + permutations


@pytest.mark.parametrize("policy,flag", [("balanced", 0), ("scheme2", spm.SPM_POLICY_SCHEME2)])
def test_repartition_keeps_copies_and_matches_oracle(policy, flag):
    """P2 re-run for new partition counts (smaller, larger than the plan was
    built with, and back): partitions bit-exact against the oracle's rule,
    MTTKRP within tolerance for every mode."""
    dims = (300, 120, 77)
    _, idx, vals = synth.coo_random(dims, 25000, seed=21)
    Y = synth.factors(dims, 32, seed=22)
    plan, _, dfac = run_all_modes(dims, idx, vals, Y, flags=flag | spm.SPM_KAPPA(16))
    for k in (3, 200, 1, 16, 1000):
        spm.spmttkrp_plan_repartition(plan, k)
        check_copies(plan, idx, kappa=k, policy=policy)
        for d in range(3):
            out = torch.full((dims[d], 32), float("nan"), device="cuda")
            spm.spmttkrp_run(plan, d, dfac, out)
            ref = check_mode_elementwise(out.cpu().numpy(), dims, idx, vals, Y, d)
            assert rel(out.cpu().numpy(), ref) < TOL
    assert spm.spmttkrp_plan_status(plan) == 0


def test_repartition_rejects_scheme1_and_bad_counts():
    dims = (50, 40, 30)
    _, idx, vals = synth.coo_random(dims, 2000, seed=3)
    Y = synth.factors(dims, 16, seed=3)
    p1, _, _ = run_all_modes(dims, idx, vals, Y, flags=spm.SPM_POLICY_SCHEME1)
    with pytest.raises(spm.SpmError) as e:
        spm.spmttkrp_plan_repartition(p1, 8)
    assert e.value.status == 7
    p0, _, _ = run_all_modes(dims, idx, vals, Y)
    with pytest.raises(spm.SpmError) as e:
        spm.spmttkrp_plan_repartition(p0, 70000)
    assert e.value.status == 1


def test_plan_autotune_picks_a_candidate_and_keeps_parity():
    dims = (3000, 800, 150)
    _, idx, vals = synth.coo_distinct(dims, 200000, (1.2, 1.2, None), seed=31)
    Y = synth.factors(dims, 32, seed=31)
    plan, _, dfac = run_all_modes(dims, idx, vals, Y)
    sms = spm.spm_device_sm_count()
    chosen, ms = spm.spmttkrp_plan_autotune(plan, dfac, [sms, 2 * sms, 7], reps=2)
    assert chosen in (sms, 2 * sms, 7) and all(m > 0 for m in ms)
    check_copies(plan, idx, kappa=chosen)
    for d in range(3):
        out = torch.full((dims[d], 32), float("nan"), device="cuda")
        spm.spmttkrp_run(plan, d, dfac, out)
        ref = check_mode_elementwise(out.cpu().numpy(), dims, idx, vals, Y, d)
        assert rel(out.cpu().numpy(), ref) < TOL
    chosen2, ms2 = spm.spmttkrp_plan_autotune(plan, dfac)  # default candidates
    assert chosen2 in (sms, 2 * sms) and len(ms2) == 2
    assert spm.spmttkrp_plan_status(plan) == 0
