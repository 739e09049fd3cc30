"""GPU tests of the batched CP-ALS engine (spm_batch_*).

A batch runs every tensor's sweep with its own plan, arithmetic and
summation order, only the launches are shared; so each tensor's factors,
weights and fit after S batched sweeps are bitwise those of S cpd_als_step
calls on it alone, whatever else is in the batch.  The single-tensor path is
itself checked against the FP64 oracle (test_gpu_als.py); one tensor here is
checked against the oracle too.
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


# (dims, nnz, R, seed): mixed mode counts, ranks and sizes; some tensors span
# many partitions (several work units, ragged tails), some fit in one.
MIX = [
    ((40, 30, 20), 900, 8, 1),
    ((300, 200, 100), 20000, 16, 2),
    ((64, 48, 32, 6), 5000, 32, 3),
    ((1000, 50, 70), 60000, 64, 4),
    ((25, 25, 25, 25), 3000, 8, 5),
    ((500, 400, 9, 3), 30000, 64, 6),
    ((33, 17, 65), 2000, 32, 7),
    ((120, 90, 60, 4), 15000, 16, 8),
    # first modes of tens of thousands of rows: many virtual row blocks in
    # every row pass of that mode, a handful in the others
    ((40000, 60, 30), 50000, 16, 9),
    ((36000, 50, 3000), 60000, 32, 10),
]


# partitions per tensor: 0 = one per SM (the default), else the count itself
KAPPAS = [0, 1, 7, 40, 3]


def make_plan(dims, nnz, R, seed, flags=0):
    _, idx, vals = synth.coo_random(dims, nnz, seed=seed)
    didx = [torch.as_tensor(c, dtype=torch.int32).cuda() for c in idx]
    dvals = torch.as_tensor(np.asarray(vals, np.float32)).cuda()
    plan = spm.spmttkrp_plan(dims, didx, dvals, R, flags)
    return plan, idx, vals


def init_factors(dims, R, seed, dtype):
    return [torch.as_tensor(f).to(dtype).cuda().contiguous()
            for f in synth.factors(dims, R, seed=100 + seed)]


def single_run(plan, fac, sweeps):
    R = plan.rank
    lam = torch.zeros(R, dtype=torch.float64, device="cuda")
    fit = torch.zeros(1, dtype=torch.float64, device="cuda")
    fits = []
    for _ in range(sweeps):
        spm.cpd_als_step(plan, fac, lam, fit)
        fits.append(fit.clone())
    assert spm.spmttkrp_plan_status(plan) == 0
    return lam, torch.cat(fits) if fits else fit


def batch_run(plans, facs, sweeps, tol=0.0, max_sweeps=None, graph=False):
    lam = torch.zeros(sum(p.rank for p in plans), dtype=torch.float64, device="cuda")
    fits = torch.zeros(len(plans), dtype=torch.float64, device="cuda")
    B = spm.spm_batch_create(plans, facs, lam, fits, tol=tol,
                             max_sweeps=max_sweeps or sweeps)
    if graph:
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                spm.spm_batch_sweep(B)
        torch.cuda.current_stream().wait_stream(s)
        for _ in range(sweeps):
            g.replay()
    else:
        for _ in range(sweeps):
            spm.spm_batch_sweep(B)
    active, nsw = spm.spm_batch_status(B)
    for p in plans:
        assert spm.spmttkrp_plan_status(p) == 0
    return B, active, nsw


def assert_same(a, b):
    assert a.dtype == b.dtype and a.shape == b.shape
    assert torch.equal(a.view(torch.int16) if a.dtype == torch.bfloat16 else a,
                       b.view(torch.int16) if b.dtype == torch.bfloat16 else b)


@pytest.mark.parametrize("dtype,flags", [(torch.float32, spm.SPM_FACTOR_FP32),
                                         (torch.bfloat16, spm.SPM_FACTOR_BF16)])
def test_batch_bitwise_equals_single_tensor_sweeps(dtype, flags):
    S = 3
    plans, facs_b, singles = [], [], []
    for dims, nnz, R, seed in MIX:
        plan, _, _ = make_plan(dims, nnz, R, seed, flags | spm.SPM_KAPPA(KAPPAS[seed % 5]))
        plans.append(plan)
        fs = init_factors(dims, R, seed, dtype)
        fb = [f.clone() for f in fs]
        lam, fit = single_run(plan, fs, S)
        singles.append((fs, lam, fit))
        facs_b.append(fb)
    B, active, nsw = batch_run(plans, facs_b, S)
    assert nsw == [S] * len(MIX)
    assert active == [0] * len(MIX)
    for t, (fs, lam, fit) in enumerate(singles):
        for w in range(len(fs)):
            assert_same(facs_b[t][w], fs[w])
        assert torch.equal(B.lam(t), lam)
        assert B.fits[t].item() == fit[-1].item()


def test_result_same_alone_and_in_mix():
    S = 2
    plans, facs_mix = [], []
    for dims, nnz, R, seed in MIX:
        plan, _, _ = make_plan(dims, nnz, R, seed)
        plans.append(plan)
        facs_mix.append(init_factors(dims, R, seed, torch.float32))
    Bm, _, _ = batch_run(plans, facs_mix, S)
    for t in (0, 3, 5):
        dims, nnz, R, seed = MIX[t]
        fa = init_factors(dims, R, seed, torch.float32)
        Ba, _, _ = batch_run([plans[t]], [fa], S)
        for w in range(len(fa)):
            assert_same(fa[w], facs_mix[t][w])
        assert torch.equal(Ba.lam(0), Bm.lam(t))
        assert Ba.fits[0].item() == Bm.fits[t].item()


def test_batch_matches_oracle_fit_and_factors():
    dims, nnz, R, seed = (64, 48, 32, 6), 5000, 32, 3
    plan, idx, vals = make_plan(dims, nnz, R, seed)
    Y0 = synth.factors(dims, R, seed=100 + seed)
    fac = [torch.as_tensor(f).cuda().contiguous() for f in Y0]
    B, _, _ = batch_run([plan], [fac], 2)
    ofac, olam, ofit = oracle.cpd_als(dims, idx, vals, Y0, 2, prec="fp32")
    assert abs(B.fits[0].item() - ofit[-1]) < 1e-3
    for w in range(4):
        g = fac[w].double().cpu().numpy()
        assert np.linalg.norm(g - ofac[w]) / np.linalg.norm(ofac[w]) < 1e-4
    lam = B.lam(0).cpu().numpy()
    assert np.linalg.norm(lam - olam) / np.linalg.norm(olam) < 1e-4


@pytest.mark.parametrize("dims,nnz,R,seed", [MIX[8], MIX[9]])
def test_long_mode_members_match_oracle(dims, nnz, R, seed):
    """Members with a first mode of tens of thousands of rows (its row passes
    split over many virtual blocks, the other modes' over a few) after two
    batched sweeps, against the oracle's CP-ALS (Sec. II-A5) on the same FP32
    factors."""
    plan, idx, vals = make_plan(dims, nnz, R, seed)
    Y0 = synth.factors(dims, R, seed=100 + seed)
    fac = [torch.as_tensor(f).cuda().contiguous() for f in Y0]
    B, _, _ = batch_run([plan], [fac], 2)
    ofac, olam, ofit = oracle.cpd_als(dims, idx, vals, Y0, 2, prec="fp32")
    assert abs(B.fits[0].item() - ofit[-1]) < 1e-3
    for w in range(3):
        g = fac[w].double().cpu().numpy()
        assert np.linalg.norm(g - ofac[w]) / np.linalg.norm(ofac[w]) < 1e-4
    lam = B.lam(0).cpu().numpy()
    assert np.linalg.norm(lam - olam) / np.linalg.norm(olam) < 1e-4


def test_bf16_batch_matches_oracle():
    """BF16-stored factors in a batch of mixed tensors: the 3- and the 4-mode
    member after two sweeps against the oracle's CP-ALS on the same
    BF16-rounded initial factors (fit within 1e-3; factors and lambda within
    2e-3, the BF16 storage rounding -- see the served-job test)."""
    sel = [MIX[1], MIX[2], MIX[6]]
    plans, facs, inputs = [], [], []
    for dims, nnz, R, seed in sel:
        plan, idx, vals = make_plan(dims, nnz, R, seed, spm.SPM_FACTOR_BF16)
        plans.append(plan)
        facs.append(init_factors(dims, R, seed, torch.bfloat16))
        inputs.append((dims, idx, vals, R, seed))
    B, _, nsw = batch_run(plans, facs, 2)
    assert nsw == [2] * len(sel)
    for t in (0, 1):
        dims, idx, vals, R, seed = inputs[t]
        Y0 = synth.factors(dims, R, seed=100 + seed)
        ofac, olam, ofit = oracle.cpd_als(dims, idx, vals, Y0, 2, prec="bf16")
        assert abs(B.fits[t].item() - ofit[-1]) < 1e-3
        for w in range(len(dims)):
            g = facs[t][w].double().cpu().numpy()
            assert np.linalg.norm(g - ofac[w]) / np.linalg.norm(ofac[w]) < 2e-3, (t, w)
        lam = B.lam(t).cpu().numpy()
        assert np.linalg.norm(lam - olam) / np.linalg.norm(olam) < 2e-3


def test_device_side_convergence_and_graph_replay():
    """Tensors stop independently once their fit changes by less than tol;
    the replayed graph of one sweep skips converged tensors on the device.
    Each tensor's state equals the single-tensor run of the same number of
    sweeps, and the stopping sweep follows the rule applied on the host."""
    tol, cap = 1e-4, 25
    plans, facs, ref = [], [], []
    for dims, nnz, R, seed in MIX[:5]:
        plan, _, _ = make_plan(dims, nnz, R, seed)
        plans.append(plan)
        facs.append(init_factors(dims, R, seed, torch.float32))
        fs = init_factors(dims, R, seed, torch.float32)
        lam, fits = single_run(plan, [f.clone() for f in fs], cap)
        f = fits.cpu().numpy()
        stop, prev = cap, -1e300
        for s in range(cap):
            if abs(f[s] - prev) < tol:
                stop = s + 1
                break
            prev = f[s]
        ref.append(stop)
    B, active, nsw = batch_run(plans, facs, cap, tol=tol, max_sweeps=cap, graph=True)
    assert nsw == ref, (nsw, ref)
    assert active == [0] * len(plans)
    for t, (dims, nnz, R, seed) in enumerate(MIX[:5]):
        fs = init_factors(dims, R, seed, torch.float32)
        lam, fits = single_run(plans[t], fs, ref[t])
        for w in range(len(fs)):
            assert_same(facs[t][w], fs[w])
        assert torch.equal(B.lam(t), lam)
        assert B.fits[t].item() == fits[-1].item()


def test_batch_rejects_unsupported_mixes():
    p32, _, _ = make_plan((30, 20, 10), 500, 16, 1)
    pbf, _, _ = make_plan((30, 20, 10), 500, 16, 1, spm.SPM_FACTOR_BF16)
    p5, _, _ = make_plan((30, 20, 10), 500, 5, 1)
    lam = torch.zeros(64, dtype=torch.float64, device="cuda")
    fits = torch.zeros(2, dtype=torch.float64, device="cuda")
    f32 = init_factors((30, 20, 10), 16, 1, torch.float32)
    fbf = init_factors((30, 20, 10), 16, 1, torch.bfloat16)
    f5 = init_factors((30, 20, 10), 5, 1, torch.float32)
    with pytest.raises(spm.SpmError) as e:
        spm.spm_batch_create([p32, pbf], [f32, fbf], lam, fits)
    assert e.value.status == 7
    with pytest.raises(spm.SpmError) as e:
        spm.spm_batch_create([p5], [f5], lam, fits)
    assert e.value.status == 7
    with pytest.raises(spm.SpmError):
        spm.spm_batch_create([p32], [f32], lam, fits, max_sweeps=0)


def test_autotune_then_batch_matches_single_tensor_sweeps():
    """The autotuner times each candidate nonzeros-per-partition value and
    leaves the plans partitioned for the fastest; batched sweeps on the tuned
    plans equal single-tensor sweeps on the same plans bitwise."""
    plans, facs, singles = [], [], []
    for dims, nnz, R, seed in MIX:
        plan, _, _ = make_plan(dims, nnz, R, seed)
        plans.append(plan)
        facs.append(init_factors(dims, R, seed, torch.float32))
    cands = (0, 512, 4096, 1 << 15)
    chosen, ms = spm.spm_batch_autotune(plans, facs, cands, reps=2)
    assert chosen in cands
    assert all(m > 0 for m in ms)
    for t, (dims, nnz, R, seed) in enumerate(MIX):
        k = spm.binding.default_kappa() if chosen == 0 else max(1, -(-plans[t].nnz // chosen))
        off = torch.empty(k + 1, dtype=torch.int64, device="cuda")
        assert spm.spmttkrp_plan_partition(plans[t], 0, off) == k
        fs = init_factors(dims, R, seed, torch.float32)
        lam, fit = single_run(plans[t], fs, 2)
        singles.append((fs, lam, fit))
    B, _, _ = batch_run(plans, facs, 2)
    for t, (fs, lam, fit) in enumerate(singles):
        for w in range(len(fs)):
            assert_same(facs[t][w], fs[w])
        assert torch.equal(B.lam(t), lam)
