"""spmttkrp_run_all_host: MTTKRP along every mode from host buffers.  The
outputs must equal those of spmttkrp_run on device buffers bitwise, with
pinned or pageable host memory, FP32 or BF16 factors, over repeated calls."""
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


@pytest.mark.parametrize("dims,R,dtype,pinned", [
    ((3000, 800, 150), 32, torch.float32, True),
    ((3000, 800, 150), 32, torch.float32, False),
    ((200, 90, 40, 7), 64, torch.bfloat16, True),
])
def test_host_buffers_match_device_path(dims, R, dtype, pinned):
    dims, idx, vals = synth.tensor_torch(dims, 60000, 5, alpha=1.1, device="cuda", max_rounds=8)
    flags = spm.SPM_FACTOR_BF16 if dtype == torch.bfloat16 else 0
    plan = spm.spmttkrp_plan(dims, idx, vals, R, flags)
    N = len(dims)
    dev_outs = []
    for rep in range(2):
        Y = [f.to(dtype).contiguous() for f in synth.factors_torch(dims, R, 10 + rep, device="cuda")]
        ref = []
        for d in range(N):
            o = torch.empty(dims[d], R, device="cuda")
            spm.spmttkrp_run(plan, d, Y, o)
            ref.append(o)
        hY = [y.cpu() for y in Y]
        hout = [torch.full((dims[d], R), float("nan")) for d in range(N)]
        if pinned:
            hY = [y.pin_memory() for y in hY]
            hout = [o.pin_memory() for o in hout]
        spm.spmttkrp_run_all_host(plan, hY, hout)
        torch.cuda.synchronize()
        for d in range(N):
            assert torch.equal(hout[d], ref[d].cpu()), f"rep {rep} mode {d}"
        dev_outs.append(ref)
    assert spm.spmttkrp_plan_status(plan) == 0
