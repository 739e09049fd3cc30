"""Host-only entry points of the C ABI, run without a GPU: the status table
and the plan-size estimate that serving admission relies on (an explicit
partition count touches no device).  The estimate's equality with the bytes a
built plan holds is checked on the GPU (tests/test_gpu_server.py)."""
import pytest

torch = pytest.importorskip("torch")

import paper_2503_18198_gb300 as spm  # noqa: E402
from paper_2503_18198_gb300 import _build, binding  # noqa: E402

OK, INVALID, CUDA = 0, 1, 4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    _build.build()
    spm.load()


def est(dims, nnz, R, kappa=304, flags=0):
    return binding.spmttkrp_plan_bytes_estimate(dims, nnz, R, flags | binding.SPM_KAPPA(kappa))


def test_status_strings_are_distinct():
    texts = [binding.spm_status_string(s) for s in range(8)]
    assert all(texts) and len(set(texts)) == 8
    assert binding.spm_status_string(99) == "unknown status"


@pytest.mark.parametrize("dims,nnz,R", [((5,), 10, 4), ((5, 6, 7), -1, 4), ((5, 6, 7), 10, 0),
                                        ((5, 6, 7), 10, binding.SPM_MAX_RANK + 1),
                                        (tuple(range(2, 2 + binding.SPM_MAX_MODES + 1)), 10, 4)])
def test_estimate_rejects_invalid_arguments(dims, nnz, R):
    with pytest.raises(spm.SpmError) as e:
        est(dims, nnz, R)
    assert e.value.status == INVALID


def test_estimate_grows_with_the_stored_layout():
    dims3, dims4 = (100_000, 50_000, 20_000), (20_000, 20_000, 5_000, 24)
    for dims, rec in ((dims3, 16), (dims4, 32)):
        N = len(dims)
        r1, t1 = est(dims, 1_000_000, 32)
        r2, t2 = est(dims, 2_000_000, 32)
        # each of the N mode copies holds a record and a 32-bit permutation entry per nonzero
        assert r2 - r1 >= N * (rec + 4) * 1_000_000
        assert t2 >= t1 >= 0
        # rank and partition count enter through the partials and the CP-ALS workspace
        assert est(dims, 1_000_000, 64)[0] > r1
        assert est(dims, 1_000_000, 32, kappa=608)[0] > r1


def test_lean_plan_is_smaller():
    dims = (100_000, 50_000, 20_000)
    full = est(dims, 5_000_000, 32)[0]
    lean = est(dims, 5_000_000, 32, flags=binding.SPM_PLAN_LEAN)[0]
    # the lean plan keeps one record copy and 32-bit positions for the others
    assert lean < full
    assert full - lean >= 2 * (16 + 4 - 4) * 5_000_000 - 2 * 16


def test_default_partition_count_needs_a_device():
    if torch.cuda.is_available():
        pytest.skip("a device is present: SPM_KAPPA(0) resolves to its SM count")
    with pytest.raises(spm.SpmError) as e:
        binding.spmttkrp_plan_bytes_estimate((100, 100, 100), 1000, 8, 0)
    assert e.value.status == CUDA


def test_sort_scratch_follows_the_nonzeros_unless_rows_are_sorted():
    # a long mode with few nonzeros: the default policy sorts nonzeros only,
    # Scheme 1 (and the adaptive rule on a mode of >= kappa rows) also sorts
    # the rows of the longest such mode by degree
    dims, nnz = (1_000_000, 300, 200), 10_000
    small = est(dims, nnz, 16)[1]
    assert small < 40 * nnz  # keys, payloads and histograms of 10,000 entries
    for policy in (binding.SPM_POLICY_SCHEME1, binding.SPM_POLICY_ADAPTIVE):
        big = est(dims, nnz, 16, flags=policy)[1]
        assert big >= 24 * dims[0]  # two 64-bit keys and two 32-bit payloads per row
    # the adaptive rule picks Scheme 2 for every mode shorter than kappa
    assert est((200, 300, 250), nnz, 16, flags=binding.SPM_POLICY_ADAPTIVE)[1] == \
        est((200, 300, 250), nnz, 16)[1]
    assert est(dims, nnz, 16, flags=binding.SPM_POLICY_SCHEME2)[1] == small
