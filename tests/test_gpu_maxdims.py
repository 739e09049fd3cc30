"""The largest index range the ABI accepts: a mode of 2^31 - 1 rows.

Indices are int32, so a mode may have up to 2^31 - 1 rows (Sec. III-C stores
an index in as few bits as the mode needs; this build keeps 32).  Here the
4-mode tensor (2^31 - 1) x 5,000 x 7 x 2,100,000 has nonzeros at both ends of
mode 0's range and in its middle, so that
  * the copy keys need 31 + 13 + 3 + 22 = 69 bits (the radix sort splits
    them over two 64-bit words),
  * the MTTKRP of modes 1-3 gathers factor rows beyond 2^31 * R elements of
    the mode-0 factor, and
  * the MTTKRP of mode 0 stores rows that far into its output and clears
    the 2^31 - 1 - (distinct rows) rows without nonzeros.
The oracle runs on the same tensor with the mode-0 indices relabelled to
0..U-1 in increasing order and the factor rows they select: relabelling an
input mode leaves every other mode's output unchanged, and an increasing
relabelling of mode 0 leaves every copy order unchanged, so permutations are
compared bit-exactly and outputs element-wise.  Needs about 70 GB of device
memory (the mode-0 factor and output, 34 GB each at R = 4).
"""
import numpy as np
import pytest

import oracle
from parity_util import abs_inputs, assert_elementwise

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2503_18198_gb300 as spm  # noqa: E402

IMAX = 2**31 - 1
R = 4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    spm.load(build_if_missing=True)


def test_mode_of_2_31_minus_1_rows():
    torch.cuda.empty_cache()
    need = 2 * IMAX * R * 4 + (8 << 30)
    if torch.cuda.mem_get_info()[0] < need:
        pytest.skip("needs about 78 GB of free device memory")
    dims = (IMAX, 5000, 7, 2_100_000)
    g = np.random.default_rng(31)
    n = 6000
    c0 = np.concatenate([IMAX - 1 - g.integers(0, 3000, 2000), g.integers(0, 3000, 2000),
                         g.integers(0, IMAX, 2000)]).astype(np.int64)
    c0[0] = IMAX - 1
    c0[1] = 0
    idx = [c0.astype(np.int32)] + [g.integers(0, dims[w], n).astype(np.int32) for w in (1, 2, 3)]
    idx[3][2] = dims[3] - 1
    vals = g.random(n).astype(np.float32)

    gen = torch.Generator(device="cuda")
    gen.manual_seed(32)
    Y0 = torch.randn(IMAX, R, generator=gen, device="cuda", dtype=torch.float32)
    Y = [g.standard_normal((dims[w], R)).astype(np.float32) for w in (1, 2, 3)]
    dfac = [Y0] + [torch.as_tensor(y).cuda() for y in Y]

    # the relabelled tensor the oracle sees
    uniq, inv = np.unique(idx[0].astype(np.int64), return_inverse=True)
    Y0_used = Y0[torch.as_tensor(uniq).cuda()].cpu().numpy()
    dims_c = (uniq.size,) + dims[1:]
    idx_c = [inv.astype(np.int32)] + idx[1:]
    fac_c = [Y0_used] + Y
    av, af = abs_inputs(vals, fac_c)

    didx = [torch.as_tensor(c).cuda() for c in idx]
    plan = spm.spmttkrp_plan(dims, didx, torch.as_tensor(vals).cuda(), R)
    try:
        for d in range(4):
            perm = torch.empty(n, dtype=torch.int64, device="cuda")
            spm.spmttkrp_plan_permutation(plan, d, perm)
            assert np.array_equal(perm.cpu().numpy(), oracle.mode_permutation(idx_c, d)), d

        # mode 0: rows at both ends of the range, every other row exactly 0
        out0 = torch.full((IMAX, R), float("nan"), device="cuda")
        spm.spmttkrp_run(plan, 0, dfac, out0)
        torch.cuda.synchronize()
        got = out0[torch.as_tensor(uniq).cuda()].double().cpu().numpy()
        ref = oracle.mttkrp(dims_c, idx_c, vals, fac_c, 0)
        absref = oracle.mttkrp(dims_c, idx_c, av, af, 0)
        assert_elementwise(got, ref, absref, what="mode 0 rows with nonzeros")
        nonzero_rows = 0
        step = 1 << 28
        for a in range(0, IMAX, step):
            nonzero_rows += int((out0[a:a + step] != 0).any(dim=1).sum())
        assert nonzero_rows == uniq.size  # NaN fill counts as non-zero: every row was written
        del out0

        # modes 1-3 gather mode-0 rows up to 2^31 - 2
        for d in (1, 2, 3):
            out = torch.full((dims[d], R), float("nan"), device="cuda")
            spm.spmttkrp_run(plan, d, dfac, out)
            torch.cuda.synchronize()
            ref = oracle.mttkrp(dims_c, idx_c, vals, fac_c, d)
            absref = oracle.mttkrp(dims_c, idx_c, av, af, d)
            assert_elementwise(out.double().cpu().numpy(), ref, absref, what=f"mode {d}")
    finally:
        plan.destroy()
        del Y0, dfac
        torch.cuda.empty_cache()
