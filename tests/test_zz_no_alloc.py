"""The allocation-free MTTKRP entry point (spmttkrp_run_noalloc).

Some callers cannot allocate device memory while they run (a serving loop
confined to a pool sized at start-up, or code where cudaMalloc would
synchronise the device).  This entry point takes a mode copy the caller
already holds and keeps its scratch in a fixed __device__ array.  The test
calls it through the C ABI twice in a row (the second call reuses the shared
scratch) and compares each result with the plan-based spmttkrp_run on the
same tensor, within the 1e-5 relative Frobenius tolerance used by the other
MTTKRP tests (the two paths split the nonzeros differently, so the FP32 sums
are not bitwise equal), and with the FP64 oracle element by element.  The
caller's records are checked on the device before use: out-of-range indices
and records out of output-row order make the call store nothing, which
spmttkrp_noalloc_status reports.  This file is collected last.
"""
import numpy as np
import pytest

import synth
from parity_util import check_mode_elementwise

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2503_18198_gb300 as spm  # noqa: E402

TOL = 1e-5


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def records_for_mode(idx, vals, mode):
    """Record layout of the header: [c_d, other indices ascending, value
    bits, zero padding], sorted by c_d (stable)."""
    N = len(idx)
    words = 4 * ((N + 1 + 3) // 4)
    order = np.argsort(idx[mode], kind="stable")
    rec = np.zeros((len(vals), words), dtype=np.int32)
    rec[:, 0] = idx[mode][order]
    col = 1
    for w in range(N):
        if w != mode:
            rec[:, col] = idx[w][order]
            col += 1
    rec[:, N] = np.asarray(vals, np.float32)[order].view(np.int32)
    return rec


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    spm.load(build_if_missing=True)


@pytest.mark.parametrize("shape,R,nnz,flags", [
    ((3000, 2000, 500), 32, 200_000, 0),
    ((400, 300, 200, 24), 16, 50_000, 0),
    ((800, 600, 90), 64, 100_000, spm.SPM_KAPPA(37)),
])
def test_noalloc_matches_plan_twice(shape, R, nnz, flags):
    dims, idx, vals = synth.coo_distinct(shape, nnz, (1.1,) * len(shape), seed=R)
    Y = synth.factors(dims, R, seed=R)
    fac = [torch.as_tensor(f).cuda() for f in Y]
    didx = [torch.as_tensor(c).cuda() for c in idx]
    plan = spm.spmttkrp_plan(dims, didx, torch.as_tensor(vals).cuda(), R, flags)
    for mode in range(len(dims)):
        ref = torch.empty(dims[mode], R, device="cuda")
        spm.spmttkrp_run(plan, mode, fac, ref)
        rec = torch.as_tensor(records_for_mode(idx, vals, mode)).cuda()
        for _ in range(2):
            out = torch.full((dims[mode], R), float("nan"), device="cuda")
            spm.spmttkrp_run_noalloc(dims, mode, R, rec, fac, out, flags)
            assert spm.binding.spmttkrp_noalloc_status() == 0
            assert rel(out.cpu().numpy(), ref.cpu().numpy()) < TOL
        if mode == 0:
            check_mode_elementwise(out.cpu().numpy(), dims, idx, vals, Y, mode)
    plan.destroy()


def test_noalloc_rejects_bad_records_on_the_device():
    """An index outside its mode's range, or records out of output-row
    order: the call clears `out` and stores nothing else; the status query
    reports the finding; the next valid call is unaffected."""
    dims = (500, 300, 200)
    dims, idx, vals = synth.coo_distinct(dims, 20_000, (1.1, 1.1, 1.1), seed=3)
    Y = synth.factors(dims, 16, seed=3)
    fac = [torch.as_tensor(f).cuda() for f in Y]
    good = records_for_mode(idx, vals, 0)
    G = 32
    for word, value, status in ((2, dims[2], 2), (1, -1, 2), (0, dims[0] + 5, 2), (None, None, 1)):
        rec = good.copy()
        if word is None:  # two neighbouring records of different rows swapped
            k = int(np.nonzero(np.diff(good[:, 0]))[0][3])
            rec[[k, k + 1]] = rec[[k + 1, k]]
        else:
            rec[777, word] = value
        buf = torch.full((dims[0] + 2 * G, 16), 3.0, device="cuda")
        out = buf[G:G + dims[0]]
        spm.spmttkrp_run_noalloc(dims, 0, 16, torch.as_tensor(rec).cuda(), fac, out)
        assert spm.binding.spmttkrp_noalloc_status() == status
        assert torch.all(out == 0.0)
        assert torch.all(buf[:G] == 3.0) and torch.all(buf[G + dims[0]:] == 3.0)
    out = torch.empty(dims[0], 16, device="cuda")
    spm.spmttkrp_run_noalloc(dims, 0, 16, torch.as_tensor(good).cuda(), fac, out)
    assert spm.binding.spmttkrp_noalloc_status() == 0
    check_mode_elementwise(out.cpu().numpy(), dims, idx, vals, Y, 0)


def test_noalloc_rejects_oversized_scratch():
    dims = (100, 100, 100)
    rec = torch.zeros((10, 4), dtype=torch.int32, device="cuda")
    fac = [torch.zeros(100, 256, device="cuda") for _ in range(3)]
    out = torch.empty(100, 256, device="cuda")
    with pytest.raises(spm.SpmError) as e:
        spm.spmttkrp_run_noalloc(dims, 0, 256, rec, fac, out, spm.SPM_KAPPA(60000))
    assert e.value.status == 7
