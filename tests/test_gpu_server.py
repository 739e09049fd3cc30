"""GPU tests of the serving loop (spm_server_*): continuous batching of CP-ALS
jobs under a device-memory budget.

A job's result must be the same alone and in the mix: the server runs each
job's sweeps with its own plan and summation order, so its factors, weights,
fit and sweep count are bitwise those of the job served alone, and those of
cpd_als_step on a plan with the same partition count run until the same
stopping rule.  Served FP32 and BF16 jobs are also compared directly with
the FP64 oracle's CP-ALS (Sec. II-A5) at the same storage precision.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2503_18198_gb300 as spm  # noqa: E402

NPP = 1 << 13  # nonzeros per partition used by the servers below


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    spm.load(build_if_missing=True)


# (dims, nnz, R, seed): 3- and 4-mode jobs of different sizes and ranks
JOBS = [
    ((300, 200, 100), 20000, 16, 11),
    ((64, 48, 32, 6), 5000, 32, 12),
    ((1000, 50, 70), 60000, 64, 13),
    ((25, 25, 25, 25), 3000, 8, 14),
    ((500, 400, 9, 3), 30000, 64, 15),
    ((120, 90, 60), 15000, 16, 16),
]


def make_inputs(dims, nnz, R, seed, alpha=1.1):
    dims, idx, vals = synth.tensor_torch(dims, nnz, seed, alpha=alpha, device="cuda",
                                         max_rounds=8)
    init = [f.contiguous() for f in synth.factors_torch(dims, R, seed, device="cuda")]
    torch.cuda.synchronize()
    return dims, idx, vals, init


def serve(jobs, flags=0, budget=8 << 30, max_active=64, arrivals=None, tol=1e-4, cap=30):
    """Serve the jobs; arrivals[k] = the step before which job k is submitted.
    Returns per job (factors, lambda, JobInfo) and the largest usage seen."""
    S = spm.Server(budget, max_active, flags, NPP)
    arrivals = arrivals or [0] * len(jobs)
    ids = [None] * len(jobs)
    peak = 0
    step = 0
    out = {}
    while len(out) < len(jobs):
        for k, a in enumerate(arrivals):
            if a == step and ids[k] is None:
                dims, idx, vals, init, R = jobs[k]
                ids[k] = S.submit(dims, idx, vals, R, init, tol=tol, max_sweeps=cap)
        S.step()
        peak = max(peak, S.usage()[0])
        for k, j in enumerate(ids):
            if j is None or k in out:
                continue
            info = S.info(j)
            if info.state == spm.binding.SPM_JOB_DONE:
                fac, lam = S.result(j)
                out[k] = (fac, lam, info)
            elif info.state == spm.binding.SPM_JOB_FAILED:
                out[k] = (None, None, info)
        step += 1
        assert step < 10 * cap + 100
    assert S.usage()[0] == 0
    S.destroy()
    return [out[k] for k in range(len(jobs))], peak


def all_jobs():
    res = []
    for dims, nnz, R, seed in JOBS:
        d, idx, vals, init = make_inputs(dims, nnz, R, seed)
        res.append((d, idx, vals, init, R))
    return res


def bits(t):
    return t.view(torch.int16) if t.dtype == torch.bfloat16 else t


@pytest.mark.parametrize("flags", [spm.SPM_FACTOR_FP32, spm.SPM_FACTOR_BF16])
def test_result_same_alone_and_in_the_mix(flags):
    jobs = all_jobs()
    # staggered arrivals: later jobs join while earlier ones are running
    mixed, _ = serve(jobs, flags, arrivals=[0, 0, 2, 3, 3, 7])
    for k in (0, 2, 4):
        alone, _ = serve([jobs[k]], flags)
        fa, la, ia = alone[0]
        fm, lm, im = mixed[k]
        assert ia.state == im.state == spm.binding.SPM_JOB_DONE
        assert ia.sweeps == im.sweeps and ia.fit == im.fit
        for a, b in zip(fa, fm):
            assert torch.equal(bits(a), bits(b))
        assert torch.equal(la, lm)


def test_server_matches_cpd_als_step_loop():
    """Same result as cpd_als_step on a plan with the server's partition
    count, stopped by the same rule (on the host here)."""
    dims, idx, vals, init, R = all_jobs()[1]
    (fs, ls, info), = serve([(dims, idx, vals, init, R)])[0]
    kappa = max(1, -(-int(vals.numel()) // NPP))
    plan = spm.spmttkrp_plan(dims, idx, vals, R, spm.SPM_KAPPA(kappa))
    fac = [f.clone() for f in init]
    lam = torch.zeros(R, dtype=torch.float64, device="cuda")
    fit = torch.zeros(1, dtype=torch.float64, device="cuda")
    prev, n = -1e300, 0
    while True:
        spm.cpd_als_step(plan, fac, lam, fit)
        n += 1
        f = float(fit.item())
        if abs(f - prev) < 1e-4 or n >= 30:
            break
        prev = f
    assert n == info.sweeps and f == info.fit
    for a, b in zip(fac, fs):
        assert torch.equal(a, b)
    assert torch.equal(lam, ls)


def test_budget_and_running_limit_respected():
    jobs = all_jobs()
    est = [spm.spmttkrp_plan_bytes_estimate(d, int(v.numel()), R,
                                            spm.SPM_KAPPA(max(1, -(-int(v.numel()) // NPP))))
           for d, _, v, _, R in jobs]
    fac_bytes = [sum(n * R * 4 for n in d) + 8 * (R + 1) for d, _, _, _, R in jobs]
    need = [r + t + f for (r, t), f in zip(est, fac_bytes)]
    # room for the largest job plus a little: jobs must queue for memory
    budget = max(need) + min(need) // 2
    res, peak = serve(jobs, budget=budget, max_active=2)
    assert peak <= budget
    assert all(r[2].state == spm.binding.SPM_JOB_DONE for r in res)
    assert any(r[2].queued_ms > 0 for r in res)


def test_job_larger_than_budget_fails_and_others_run():
    jobs = all_jobs()[:3]
    d, _, v, _, R = jobs[2]
    r, t = spm.spmttkrp_plan_bytes_estimate(d, int(v.numel()), R,
                                            spm.SPM_KAPPA(max(1, -(-int(v.numel()) // NPP))))
    budget = r + t - 1  # job 2 can never fit, jobs 0 and 1 can
    res, _ = serve(jobs, budget=budget)
    assert res[2][2].state == spm.binding.SPM_JOB_FAILED and res[2][2].status == 3
    assert res[0][2].state == res[1][2].state == spm.binding.SPM_JOB_DONE


def test_plan_bytes_estimate_equals_plan_bytes():
    for dims, nnz, R, seed in JOBS[:4]:
        d, idx, vals, init = make_inputs(dims, nnz, R, seed)
        for flags in (0, spm.SPM_KAPPA(7)):
            plan = spm.spmttkrp_plan(d, idx, vals, R, flags)
            lam = torch.zeros(R, dtype=torch.float64, device="cuda")
            spm.cpd_als_step(plan, [f.clone() for f in init], lam)
            res, tr = spm.spmttkrp_plan_bytes_estimate(d, int(vals.numel()), R, flags)
            assert res == spm.spmttkrp_plan_bytes(plan)
            assert tr > 0


# BF16-stored factors: a factor element whose FP32 update lands within the
# GPU's accumulation error (~1e-6 relative) of a BF16 rounding boundary rounds
# the other way than the oracle's, a change of 2^-8 of that element; such
# flips, carried through the next modes' updates, keep whole factors within a
# few 1e-4 of the oracle's after a few sweeps.
FAC_TOL = {spm.SPM_FACTOR_FP32: 1e-4, spm.SPM_FACTOR_BF16: 2e-3}


@pytest.mark.parametrize("flags,prec", [(spm.SPM_FACTOR_FP32, "fp32"),
                                        (spm.SPM_FACTOR_BF16, "bf16")])
def test_served_jobs_match_oracle(flags, prec):
    """Jobs served in a staggered mix (3- and 4-mode, R = 16, 32, 64), each
    run for exactly S sweeps (tol = 0), against the oracle's CP-ALS from the
    same initial factors rounded to the same storage type: fit within 1e-3,
    lambda and every factor within FAC_TOL relative Frobenius error."""
    S = 3
    jobs = all_jobs()
    res, _ = serve(jobs, flags, arrivals=[0, 0, 1, 1, 2, 2], tol=0.0, cap=S)
    for k in (0, 1, 4):
        dims, idx, vals, init, R = jobs[k]
        fac, lam, info = res[k]
        assert info.state == spm.binding.SPM_JOB_DONE and info.sweeps == S
        ofac, olam, ofit = oracle.cpd_als(dims, [c.cpu().numpy() for c in idx],
                                          vals.cpu().numpy(), [f.cpu().numpy() for f in init],
                                          S, prec=prec)
        assert abs(info.fit - ofit[-1]) < 1e-3, (k, info.fit, ofit[-1])
        tol = FAC_TOL[flags]
        lam_h = lam.cpu().numpy()
        assert np.linalg.norm(lam_h - olam) / np.linalg.norm(olam) < tol, k
        for w in range(len(dims)):
            g = fac[w].double().cpu().numpy()
            assert np.linalg.norm(g - ofac[w]) / np.linalg.norm(ofac[w]) < tol, (k, w)
