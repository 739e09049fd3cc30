"""Failure detection without a GPU fault.

* A bounded device-side wait that nothing completes gives up, records a
  timeout that the host reads as SPM_ERR_TIMEOUT, and the context stays
  usable; the MTTKRP kernel's own record-copy waits, made to give up at
  once, leave every copy landed and no store outside (or inside) the output.
* Allocation failures are injected on the host (a fake of the failing
  cudaMalloc): every allocation point of a plan returns SPM_ERR_OOM cleanly,
  without leaking device memory, and the next plan succeeds.
* Non-finite factors make the ALS normal equations fail: SPM_ERR_NUMERIC,
  in cpd_als_step and for a served job, whose neighbours finish unaffected.
"""
import numpy as np
import pytest

import oracle
import synth
from parity_util import check_mode_elementwise

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2503_18198_gb300 as spm  # noqa: E402

SPM_ERR_OOM, SPM_ERR_NUMERIC, SPM_ERR_TIMEOUT = 3, 5, 6


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    spm.load(build_if_missing=True)
    yield
    spm.binding.spm_inject_alloc_failure(-1)


def small_problem(R=16, seed=5):
    dims = (120, 80, 60)
    _, idx, vals = synth.coo_random(dims, 6000, seed=seed)
    Y = synth.factors(dims, R, seed=seed)
    didx = [torch.as_tensor(c).cuda() for c in idx]
    dvals = torch.as_tensor(vals).cuda()
    return dims, idx, vals, Y, didx, dvals


def test_bounded_wait_times_out_and_context_stays_usable():
    for limit in (1, 64, 4096):
        assert spm.binding.spm_selftest_wait_timeout(limit) == SPM_ERR_TIMEOUT
    dims, idx, vals, Y, didx, dvals = small_problem()
    plan = spm.spmttkrp_plan(dims, didx, dvals, 16)
    fac = [torch.as_tensor(f).cuda() for f in Y]
    out = torch.empty(dims[0], 16, device="cuda")
    spm.spmttkrp_run(plan, 0, fac, out)
    ref = oracle.mttkrp(dims, idx, vals, Y, 0)
    assert np.linalg.norm(out.cpu().numpy() - ref) / np.linalg.norm(ref) < 1e-5
    assert spm.spmttkrp_plan_status(plan) == 0


@pytest.mark.parametrize("dims,R,alphas,kappa", [
    ((3000, 2000, 500), 32, (1.2, 1.2, 1.2), 0),      # default plan, Zipf heads
    ((400, 300, 200, 24), 16, (1.0, 1.0, None, None), 37),
])
def test_mttkrp_kernel_wait_timeout_stores_nothing(dims, R, alphas, kappa):
    """The MTTKRP kernel's own record-copy waits made to give up at once
    (no poll at all): each warp waits for the copies it already issued,
    the block skips its merge and every store, the host reads
    SPM_ERR_TIMEOUT, guard rows around the output keep their contents, and
    the next ordinary run on the same plan matches the oracle."""
    dims, idx, vals = synth.coo_distinct(dims, 150_000, alphas, seed=R)
    Y = synth.factors(dims, R, seed=R)
    fac = [torch.as_tensor(f).cuda() for f in Y]
    didx = [torch.as_tensor(c).cuda() for c in idx]
    plan = spm.spmttkrp_plan(dims, didx, torch.as_tensor(vals).cuda(), R, spm.SPM_KAPPA(kappa))
    G = 64  # guard rows before and after the output
    for d in range(len(dims)):
        buf = torch.full((dims[d] + 2 * G, R), 7.0, device="cuda")
        out = buf[G:G + dims[d]]
        assert spm.binding.spm_selftest_mttkrp_timeout(plan, d, fac, out) == SPM_ERR_TIMEOUT
        torch.cuda.synchronize()
        assert torch.all(buf[:G] == 7.0) and torch.all(buf[G + dims[d]:] == 7.0)
        got = out.cpu().numpy()
        nonempty = np.bincount(idx[d], minlength=dims[d]) > 0
        assert np.all(got[~nonempty] == 0.0)  # the empty-row clear still ran
        assert np.all(got[nonempty] == 7.0)   # no row of a timed-out block was stored
        spm.spmttkrp_run(plan, d, fac, out)
        assert spm.spmttkrp_plan_status(plan) == 0
        ref = check_mode_elementwise(out.cpu().numpy(), dims, idx, vals, Y, d)
        assert np.linalg.norm(out.cpu().numpy() - ref) / np.linalg.norm(ref) < 1e-5
        assert torch.all(buf[:G] == 7.0) and torch.all(buf[G + dims[d]:] == 7.0)
    plan.destroy()


def test_injected_allocation_failures_are_clean():
    dims, idx, vals, Y, didx, dvals = small_problem()
    # warm-up: the first launches of each kernel load its module and reserve
    # its local memory; the baseline is taken after that
    plan = spm.spmttkrp_plan(dims, didx, dvals, 16)
    spm.cpd_als_step(plan, [torch.as_tensor(f).cuda() for f in Y],
                     torch.zeros(16, dtype=torch.float64, device="cuda"))
    plan.destroy()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    failures = 0
    for k in range(40):
        spm.binding.spm_inject_alloc_failure(k)
        try:
            plan = spm.spmttkrp_plan(dims, didx, dvals, 16)
        except spm.SpmError as e:
            assert e.status == SPM_ERR_OOM
            failures += 1
            continue
        # the plan's own allocations are done: the fault (if still armed) hits
        # the CP-ALS workspace, allocated by the first sweep
        fac = [torch.as_tensor(f).cuda() for f in Y]
        lam = torch.zeros(16, dtype=torch.float64, device="cuda")
        try:
            spm.cpd_als_step(plan, fac, lam)
        except spm.SpmError as e:
            assert e.status == SPM_ERR_OOM
            failures += 1
        plan.destroy()
        spm.binding.spm_inject_alloc_failure(-1)
    assert failures >= 20  # every allocation point of the plan and its workspace
    spm.binding.spm_inject_alloc_failure(-1)
    plan = spm.spmttkrp_plan(dims, didx, dvals, 16)
    fac = [torch.as_tensor(f).cuda() for f in Y]
    lam = torch.zeros(16, dtype=torch.float64, device="cuda")
    fit = torch.zeros(1, dtype=torch.float64, device="cuda")
    spm.cpd_als_step(plan, fac, lam, fit)
    _, _, ofit = oracle.cpd_als(dims, idx, vals, Y, 1, prec="fp32")
    assert abs(float(fit.item()) - ofit[0]) < 1e-3
    plan.destroy()
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert abs(free1 - free0) < (16 << 20)  # nothing of the failed plans stays allocated


def test_nonfinite_factor_reports_numeric_error():
    dims, idx, vals, Y, didx, dvals = small_problem()
    plan = spm.spmttkrp_plan(dims, didx, dvals, 16)
    Y[1][3, 2] = np.nan
    fac = [torch.as_tensor(f).cuda() for f in Y]
    lam = torch.zeros(16, dtype=torch.float64, device="cuda")
    spm.cpd_als_step(plan, fac, lam)
    assert spm.spmttkrp_plan_status(plan) == SPM_ERR_NUMERIC
    # the status is cleared once read; the plan works again on finite factors
    Y[1][3, 2] = 0.5
    fac = [torch.as_tensor(f).cuda() for f in Y]
    spm.cpd_als_step(plan, fac, lam)
    assert spm.spmttkrp_plan_status(plan) == 0


def test_served_job_with_nonfinite_factors_fails_alone():
    jobs = []
    for seed in (21, 22, 23):
        dims, idx, vals = synth.coo_random((200, 150, 90), 20000, seed=seed)[0:3]
        init = [f.contiguous() for f in synth.factors_torch(dims, 16, seed, device="cuda")]
        jobs.append((dims, [torch.as_tensor(c).cuda() for c in idx],
                     torch.as_tensor(vals).cuda(), init))
    jobs[1][3][1][5, 1] = float("inf")  # factor 1 enters the first update (mode 0)
    torch.cuda.synchronize()

    def serve(js):
        S = spm.Server(4 << 30, 8, 0, 1 << 12)
        ids = [S.submit(d, i, v, 16, f, tol=1e-4, max_sweeps=10) for d, i, v, f in js]
        for _ in range(40):
            S.step()
            if all(S.info(j).state >= spm.binding.SPM_JOB_DONE for j in ids):
                break
        infos = [S.info(j) for j in ids]
        res = [S.result(j) if inf.state == spm.binding.SPM_JOB_DONE else None
               for j, inf in zip(ids, infos)]
        assert S.usage()[0] == 0
        S.destroy()
        return infos, res
    infos, res = serve(jobs)
    assert infos[1].state == spm.binding.SPM_JOB_FAILED and infos[1].status == SPM_ERR_NUMERIC
    for k in (0, 2):
        assert infos[k].state == spm.binding.SPM_JOB_DONE
        alone_info, alone_res = serve([jobs[k]])
        assert alone_info[0].fit == infos[k].fit and alone_info[0].sweeps == infos[k].sweeps
        for a, b in zip(alone_res[0][0], res[k][0]):
            assert torch.equal(a, b)
