"""Fibre-layout copies (SPM_PLAN_FIBRE): each 3-mode copy stored as fibre
headers {c_d, c_a} followed by their nonzeros {c_b, value}, the MTTKRP
gathering Y_a once per fibre.

Checked against the FP64 oracle and against independent definitions:
  * every mode's output element by element (|err| <= 1e-5 * sum|terms|) and
    within 1e-5 relative Frobenius error, FP32 and BF16 factors (the latter
    against the oracle on the same BF16 values);
  * the fibre count of every copy equals the number of distinct (c_d, c_a)
    pairs (a Python set over the input) -- bit-exact integer structure;
  * permutations and partitions are the record layout's, bit-exactly;
  * CP-ALS on a fibre plan against the oracle's CP-ALS;
  * the kernel's bounded waits made to give up store nothing;
  * edge cases: empty tensor, one nonzero, tiny output modes (every partition
    on a few rows), empty rows, many partitions (empty units), long fibres.
"""
import numpy as np
import pytest

import oracle
import synth
from parity_util import check_mode_elementwise

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2503_18198_gb300 as spm  # noqa: E402

TOL = 1e-5
FIBRE = spm.SPM_PLAN_FIBRE


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    spm.load(build_if_missing=True)


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def make(dims, idx, vals, R, flags, dtype=torch.float32, seed=0):
    didx = [torch.as_tensor(np.asarray(c, np.int32)).cuda() for c in idx]
    dvals = torch.as_tensor(np.asarray(vals, np.float32)).cuda()
    plan = spm.spmttkrp_plan(dims, didx, dvals, R, flags)
    Y = synth.factors(dims, R, seed=seed)
    fac = [torch.as_tensor(f).to(dtype).cuda().contiguous() for f in Y]
    return plan, Y, fac


def run(plan, fac, dims, R):
    outs = []
    for d in range(3):
        out = torch.full((dims[d], R), float("nan"), device="cuda")
        spm.spmttkrp_run(plan, d, fac, out)
        outs.append(out)
    torch.cuda.synchronize()
    return [o.cpu().numpy() for o in outs]


def distinct_fibres(idx, d):
    a = [w for w in range(3) if w != d][0]
    return len(set(zip(idx[d].tolist(), idx[a].tolist())))


CASES = [
    # dims, nnz, alphas, R, kappa (0 = default)
    ((3000, 2000, 500), 200_000, (1.2, 1.2, 1.2), 32, 0),     # Zipf heads: long fibres
    ((3000, 2000, 500), 200_000, (1.2, 1.2, 1.2), 16, 37),
    ((800, 600, 90), 100_000, (1.1, 1.1, None), 64, 0),
    ((1000, 12, 11), 4000, (None, None, None), 32, 152),      # empty rows in mode 0
    ((3, 1000, 5), 6000, (None, None, None), 32, 152),        # tiny output mode
    ((50, 40, 30), 700, (None, None, None), 16, 300),         # more units than nonzeros
    ((2000, 3, 2), 9000, (1.3, None, None), 64, 7),           # fibres of up to thousands
]


@pytest.mark.parametrize("dims,nnz,alphas,R,kappa", CASES)
def test_fibre_plan_matches_oracle_and_record_layout(dims, nnz, alphas, R, kappa):
    dims, idx, vals = synth.coo_distinct(dims, nnz, alphas, seed=R + kappa)
    plan, Y, fac = make(dims, idx, vals, R, FIBRE | spm.SPM_KAPPA(kappa), seed=R)
    ref_plan, _, _ = make(dims, idx, vals, R, spm.SPM_KAPPA(kappa), seed=R)
    outs = run(plan, fac, dims, R)
    k = kappa or spm.binding.default_kappa()
    for d in range(3):
        ref = check_mode_elementwise(outs[d], dims, idx, vals, Y, d)
        assert rel(outs[d], ref) < TOL, f"mode {d}"
        assert spm.spmttkrp_plan_fibre_count(plan, d) == distinct_fibres(idx, d)
        # same P1 order and P2 partition as the record layout (bit-exact)
        for fn, size in ((spm.spmttkrp_plan_permutation, plan.nnz),):
            a = torch.empty(size, dtype=torch.int64, device="cuda")
            b = torch.empty(size, dtype=torch.int64, device="cuda")
            fn(plan, d, a)
            fn(ref_plan, d, b)
            assert torch.equal(a, b)
        assert np.array_equal(a.cpu().numpy(), oracle.mode_permutation(idx, d))
        oa = torch.empty(k + 1, dtype=torch.int64, device="cuda")
        ob = torch.empty(k + 1, dtype=torch.int64, device="cuda")
        spm.spmttkrp_plan_partition(plan, d, oa)
        spm.spmttkrp_plan_partition(ref_plan, d, ob)
        assert torch.equal(oa, ob)
    # repeated runs are bitwise identical
    again = run(plan, fac, dims, R)
    assert all(np.array_equal(x, y) for x, y in zip(outs, again))
    assert spm.spmttkrp_plan_status(plan) == 0


@pytest.mark.parametrize("R", [16, 32, 64])
def test_fibre_plan_bf16_factors(R):
    dims, idx, vals = synth.coo_distinct((3001, 203, 97), 30_000, (1.1, 1.1, None), seed=R)
    plan, Y, fac = make(dims, idx, vals, R, FIBRE | spm.SPM_FACTOR_BF16, torch.bfloat16, seed=R)
    outs = run(plan, fac, dims, R)
    Yb = [f.float().cpu().numpy() for f in fac]
    for d in range(3):
        ref = check_mode_elementwise(outs[d], dims, idx, vals, Yb, d)
        assert rel(outs[d], ref) < TOL
        assert rel(outs[d], oracle.mttkrp(dims, idx, vals, Y, d)) < 2e-2


def test_fibre_plan_bytes():
    dims, idx, vals = synth.coo_distinct((3000, 2000, 500), 200_000, (1.2, 1.2, 1.2), seed=3)
    a, _, _ = make(dims, idx, vals, 32, FIBRE)
    b, _, _ = make(dims, idx, vals, 32, 0)
    # per mode: a 16-byte record per nonzero (+256 padding) becomes an 8-byte
    # entry per nonzero and per fibre (+2 padding entries) plus a 32-byte
    # table entry per work unit; the fibre plan has kappa * 32 * 128 / R work
    # units (8-byte offsets each) against kappa * SPM_UNITS_PER_PARTITION(R)
    k = spm.binding.default_kappa()
    P, P_rec = k * 32 * 128 // 32, k * spm.SPM_UNITS_PER_PARTITION(32)
    saved = sum((16 * a.nnz + 256) - 8 * (a.nnz + spm.spmttkrp_plan_fibre_count(a, d) + 2)
                - 32 * P - 8 * (P - P_rec) for d in range(3))
    assert spm.spmttkrp_plan_bytes(b) - spm.spmttkrp_plan_bytes(a) == saved
    est, _ = spm.spmttkrp_plan_bytes_estimate(dims, a.nnz, 32, FIBRE)
    assert est >= spm.spmttkrp_plan_bytes(a)  # an upper bound for fibre plans


def test_fibre_plan_cp_als_matches_oracle():
    dims, idx, vals = synth.coo_distinct((300, 200, 100), 20_000, (1.1, 1.1, 1.1), seed=5)
    plan, Y, fac = make(dims, idx, vals, 16, FIBRE, seed=5)
    lam = torch.zeros(16, dtype=torch.float64, device="cuda")
    fit = torch.zeros(1, dtype=torch.float64, device="cuda")
    fits = []
    for _ in range(3):
        spm.cpd_als_step(plan, fac, lam, fit)
        fits.append(float(fit.item()))
    assert spm.spmttkrp_plan_status(plan) == 0
    ofac, olam, ofit = oracle.cpd_als(dims, idx, vals, Y, 3, prec="fp32")
    assert np.all(np.abs(np.array(fits) - ofit) < 1e-3)
    for w in range(3):
        assert rel(fac[w].cpu().numpy(), ofac[w]) < 1e-4
    assert rel(lam.cpu().numpy(), olam) < 1e-4


def test_fibre_plan_wait_timeout_stores_nothing():
    dims, idx, vals = synth.coo_distinct((3000, 2000, 500), 100_000, (1.2, 1.2, 1.2), seed=9)
    plan, Y, fac = make(dims, idx, vals, 32, FIBRE, seed=9)
    G = 32
    for d in range(3):
        buf = torch.full((dims[d] + 2 * G, 32), 5.0, device="cuda")
        out = buf[G:G + dims[d]]
        assert spm.binding.spm_selftest_mttkrp_timeout(plan, d, fac, out) == 6
        nonempty = np.bincount(idx[d], minlength=dims[d]) > 0
        got = out.cpu().numpy()
        assert np.all(got[nonempty] == 5.0) and np.all(got[~nonempty] == 0.0)
        assert torch.all(buf[:G] == 5.0) and torch.all(buf[G + dims[d]:] == 5.0)
        spm.spmttkrp_run(plan, d, fac, out)
        check_mode_elementwise(out.cpu().numpy(), dims, idx, vals, Y, d)


def test_fibre_plan_edge_cases_and_rejections():
    dims = (5, 4, 3)
    plan, Y, fac = make(dims, [np.zeros(0, np.int32)] * 3, np.zeros(0, np.float32), 32, FIBRE)
    assert all(np.all(o == 0) for o in run(plan, fac, dims, 32))
    assert all(spm.spmttkrp_plan_fibre_count(plan, d) == 0 for d in range(3))
    idx = [np.array([4], np.int32), np.array([0], np.int32), np.array([2], np.int32)]
    plan, Y, fac = make(dims, idx, np.array([2.0], np.float32), 32, FIBRE)
    outs = run(plan, fac, dims, 32)
    for d in range(3):
        check_mode_elementwise(outs[d], dims, idx, [2.0], Y, d)
    # outside the fibre kernel's shapes, or with features it does not support
    g = np.random.default_rng(0)
    idx4 = [g.integers(0, 5, 50).astype(np.int32) for _ in range(4)]
    for d4, ix, R, extra in (((5, 5, 5, 5), idx4, 32, 0), (dims, idx, 8, 0),
                             (dims, idx, 32, spm.SPM_PLAN_LEAN),
                             (dims, idx, 32, spm.SPM_POLICY_SCHEME1)):
        with pytest.raises(spm.SpmError) as e:
            make(d4, ix, np.ones(ix[0].size, np.float32), R, FIBRE | extra)
        assert e.value.status == 7
    plan, Y, fac = make(dims, idx, np.array([2.0], np.float32), 32, FIBRE)
    with pytest.raises(spm.SpmError) as e:
        spm.spmttkrp_plan_repartition(plan, 3)
    assert e.value.status == 7
    with pytest.raises(spm.SpmError) as e:
        spm.spmttkrp_plan_fibre_count(make(dims, idx, np.array([2.0], np.float32), 32, 0)[0], 0)
    assert e.value.status == 7
