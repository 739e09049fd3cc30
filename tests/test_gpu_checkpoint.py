"""Checkpoint / resume of CP-ALS.

The state of a CP-ALS run is its factors, lambda, sweep count and last fit.
A run resumed from a copy of that state must continue bitwise as the
uninterrupted run: single-tensor runs (factors restored into new buffers, or
into the same buffers followed by cpd_als_reset) and served jobs
(spm_server_snapshot, then spm_server_resume on a fresh server).
"""
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2503_18198_gb300 as spm  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    spm.load(build_if_missing=True)


def problem(seed=3, dims=(400, 250, 120), nnz=30000, R=16):
    dims, idx, vals = synth.tensor_torch(dims, nnz, seed, alpha=1.1, device="cuda", max_rounds=8)
    init = [f.contiguous() for f in synth.factors_torch(dims, R, seed, device="cuda")]
    torch.cuda.synchronize()
    return dims, idx, vals, init, R


def sweeps(plan, fac, lam, fit, n):
    for _ in range(n):
        spm.cpd_als_step(plan, fac, lam, fit)
    torch.cuda.synchronize()


def test_single_tensor_resume_is_bitwise():
    dims, idx, vals, init, R = problem()
    plan = spm.spmttkrp_plan(dims, idx, vals, R)
    z = lambda: (torch.zeros(R, dtype=torch.float64, device="cuda"),  # noqa: E731
                 torch.zeros(1, dtype=torch.float64, device="cuda"))
    ref = [f.clone() for f in init]
    lam_ref, fit_ref = z()
    sweeps(plan, ref, lam_ref, fit_ref, 6)

    # interrupted after 3 sweeps, resumed from copies in new buffers
    run = [f.clone() for f in init]
    lam, fit = z()
    sweeps(plan, run, lam, fit, 3)
    saved = [f.clone() for f in run]
    resumed = [f.clone() for f in saved]
    sweeps(plan, resumed, lam, fit, 3)
    for a, b in zip(resumed, ref):
        assert torch.equal(a, b)
    assert torch.equal(lam, lam_ref) and torch.equal(fit, fit_ref)

    # restored into the same buffers after other work: needs cpd_als_reset
    sweeps(plan, resumed, lam, fit, 1)           # the buffers move on
    for dst, src in zip(resumed, saved):
        dst.copy_(src)
    spm.cpd_als_reset(plan)
    sweeps(plan, resumed, lam, fit, 3)
    for a, b in zip(resumed, ref):
        assert torch.equal(a, b)
    assert torch.equal(fit, fit_ref)
    assert spm.spmttkrp_plan_status(plan) == 0


@pytest.mark.parametrize("flags", [spm.SPM_FACTOR_FP32, spm.SPM_FACTOR_BF16])
def test_served_job_resume_is_bitwise(flags):
    dims, idx, vals, init, R = problem(seed=9)

    def finish(S, j):
        for _ in range(100):
            S.step()
            if S.info(j).state != spm.binding.SPM_JOB_RUNNING and \
               S.info(j).state != spm.binding.SPM_JOB_QUEUED:
                break
        info = S.info(j)
        assert info.state == spm.binding.SPM_JOB_DONE
        fac, lam = S.result(j)
        return info, fac, lam

    S = spm.Server(2 << 30, 4, flags, 1 << 12)
    j = S.submit(dims, idx, vals, R, init, tol=1e-7, max_sweeps=12)
    info_ref, fac_ref, lam_ref = finish(S, j)
    S.destroy()
    assert info_ref.sweeps > 4

    S = spm.Server(2 << 30, 4, flags, 1 << 12)
    j = S.submit(dims, idx, vals, R, init, tol=1e-7, max_sweeps=12)
    for _ in range(4):
        S.step()
    assert S.info(j).state == spm.binding.SPM_JOB_RUNNING
    snap_fac, snap_lam, done, prev_fit = S.snapshot(j)
    assert 0 < done < info_ref.sweeps
    S.destroy()  # the interruption

    S = spm.Server(2 << 30, 4, flags, 1 << 12)
    j = S.submit(dims, idx, vals, R, [f.float().contiguous() for f in snap_fac], tol=1e-7,
                 max_sweeps=12, resume=(done, prev_fit))
    info, fac, lam = finish(S, j)
    S.destroy()
    assert info.sweeps == info_ref.sweeps and info.fit == info_ref.fit
    for a, b in zip(fac, fac_ref):
        assert torch.equal(a.view(torch.int16) if a.dtype == torch.bfloat16 else a,
                           b.view(torch.int16) if b.dtype == torch.bfloat16 else b)
    assert torch.equal(lam, lam_ref)
