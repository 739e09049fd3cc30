"""GPU parity of cpd_als_step (one CP-ALS sweep per call) against the oracle.

Tolerances: the fit after the same number of sweeps within 1e-3 of the FP64
oracle's (the oracle rounds its factors to the same storage type after every
update); factors after one sweep within 1e-4 relative Frobenius error (FP32
MTTKRP and FP32 storage, FP64 Cholesky); exact recovery of a rank-R tensor.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2503_18198_gb300 as spm  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    spm.load(build_if_missing=True)


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def gpu_als(dims, idx, vals, Y0, sweeps, flags=0, dtype=torch.float32):
    didx = [torch.as_tensor(c, dtype=torch.int32).cuda() for c in idx]
    dvals = torch.as_tensor(np.asarray(vals, np.float32)).cuda()
    R = Y0[0].shape[1]
    plan = spm.spmttkrp_plan(dims, didx, dvals, R, flags)
    fac = [torch.as_tensor(np.asarray(f, np.float32)).to(dtype).cuda().contiguous() for f in Y0]
    lam = torch.zeros(R, dtype=torch.float64, device="cuda")
    fit = torch.zeros(1, dtype=torch.float64, device="cuda")
    fits = []
    for _ in range(sweeps):
        spm.cpd_als_step(plan, fac, lam, fit)
        fits.append(float(fit.item()))
    assert spm.spmttkrp_plan_status(plan) == 0
    return plan, [f.float().cpu().numpy() for f in fac], lam.cpu().numpy(), np.array(fits)


def test_plain_workload_five_sweeps():
    dims, idx, vals, R, Y = synth.preset("plain")
    _, fac1, lam1, fit1 = gpu_als(dims, idx, vals, Y, 1)
    ofac1, olam1, ofit1 = oracle.cpd_als(dims, idx, vals, Y, 1, prec="fp32")
    for d in range(3):
        assert rel(fac1[d], ofac1[d]) < 1e-4
    assert rel(lam1, olam1) < 1e-4
    _, fac5, lam5, fit5 = gpu_als(dims, idx, vals, Y, 5)
    _, _, ofit5 = oracle.cpd_als(dims, idx, vals, Y, 5, prec="fp32")
    assert np.all(np.abs(fit5 - ofit5) < 1e-3), (fit5, ofit5)


@pytest.mark.parametrize("R", [5, 8, 13, 16])
def test_narrow_rank_rows_with_tails_and_empty_rows(R):
    """Ranks <= 16 put 2 or 4 rows in one warp instruction of the row solve:
    ragged ranks (lanes past R idle), row counts that are not a multiple of
    the row group, and empty rows (Zipf coordinates on dims larger than the
    rows the nonzeros reach) skipped by whole groups."""
    dims, idx, vals = synth.coo_distinct((1001, 707, 333), 20000, (1.3, 1.3, None), seed=40 + R)
    assert any(len(np.unique(c)) < n for c, n in zip(idx, dims))  # some mode has empty rows
    Y = synth.factors(dims, R, seed=40 + R)
    _, fac1, lam1, fit1 = gpu_als(dims, idx, vals, Y, 1)
    ofac1, olam1, ofit1 = oracle.cpd_als(dims, idx, vals, Y, 1, prec="fp32")
    for d in range(3):
        assert rel(fac1[d], ofac1[d]) < 1e-4
    assert rel(lam1, olam1) < 1e-4
    assert abs(fit1[0] - ofit1[0]) < 1e-3


@pytest.mark.parametrize("R,block,dims", [(3, 3, (10, 11, 12)), (4, 3, (12, 13, 14))])
def test_exact_recovery(R, block, dims):
    """The GPU's factors reconstruct an exactly rank-R tensor (residual taken
    densely on the host in FP64 from the GPU's lambda and factors).  The
    GPU's own fit value agrees with the oracle's within 1e-3: near fit = 1
    the fit identity subtracts nearly equal terms built from the FP32
    MTTKRP, so it resolves the fit only to about sqrt(eps_fp32)."""
    dims, idx, vals, true = synth.rank_r_blocks(dims, R, block, seed=4)
    X = np.zeros(dims)
    for k in range(vals.size):
        X[idx[0][k], idx[1][k], idx[2][k]] += vals[k]
    best = 0.0
    for seed in range(4):
        Y0 = synth.factors(dims, R, seed=seed)
        _, fac, lam, fit = gpu_als(dims, idx, vals, Y0, 60, flags=spm.SPM_KAPPA(5))
        _, _, ofit = oracle.cpd_als(dims, idx, vals, Y0, 60, prec="fp32")
        assert abs(fit[-1] - ofit[-1]) < 1e-3
        Xh = np.einsum("r,ir,jr,kr->ijk", lam, *[f.astype(np.float64) for f in fac])
        best = max(best, 1.0 - np.linalg.norm(X - Xh) / np.linalg.norm(X))
    assert best > 0.9999


def test_four_modes_and_kappa():
    dims, idx, vals = synth.coo_distinct((40, 30, 20, 6), 3000, (1.0, 1.0, 1.0, None), seed=8,
                                         values="lognormal")
    Y = synth.factors(dims, 8, seed=8)
    _, fac, lam, fit = gpu_als(dims, idx, vals, Y, 3, flags=spm.SPM_KAPPA(7))
    ofac, olam, ofit = oracle.cpd_als(dims, idx, vals, Y, 3, prec="fp32")
    assert np.all(np.abs(fit - ofit) < 1e-3)


@pytest.mark.parametrize("R", [16, 32, 64])
def test_bf16_factors(R):
    dims, idx, vals = synth.coo_distinct((300, 200, 100), 8000, (1.1, 1.1, 1.1), seed=R)
    Y = synth.factors(dims, R, seed=R)
    Yb = [oracle.store_round(f, "bf16") for f in Y]
    _, fac, lam, fit = gpu_als(dims, idx, vals, Yb, 4, flags=spm.SPM_FACTOR_BF16,
                               dtype=torch.bfloat16)
    _, _, ofit = oracle.cpd_als(dims, idx, vals, Yb, 4, prec="bf16")
    assert np.all(np.abs(fit - ofit) < 1e-3), (fit, ofit)


def test_singular_system_reports_numeric_error():
    dims = (6, 5, 4)
    g = np.random.default_rng(1)
    idx = [g.integers(0, n, 40).astype(np.int32) for n in dims]
    vals = g.random(40).astype(np.float32)
    Y = [np.ones((n, 3), np.float32) for n in dims]   # identical columns
    didx = [torch.as_tensor(c).cuda() for c in idx]
    plan = spm.spmttkrp_plan(dims, didx, torch.as_tensor(vals).cuda(), 3)
    fac = [torch.as_tensor(f).cuda() for f in Y]
    before = [f.clone() for f in fac]
    lam = torch.zeros(3, dtype=torch.float64, device="cuda")
    spm.cpd_als_step(plan, fac, lam, None)
    assert spm.spmttkrp_plan_status(plan) == 5
    # the failing mode left the factors untouched
    assert all(torch.equal(a, b) for a, b in zip(fac, before))
    # the status is cleared once read
    assert spm.spmttkrp_plan_status(plan) == 0
