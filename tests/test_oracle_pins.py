"""Pins of the FP64 oracle against facts that do not go through its code.

Each test checks one oracle routine against something the paper or the
mathematics fixes: a hand-worked example, dense brute force with an explicit
Khatri-Rao product (Eq. 1 in the paper's operand order and in Kolda's), the
rank-1 closed form, invariants (linearity, duplicates, input order, the
mode-independent inner product), sorting by an independent implementation,
the partition formulas, the normal equations of the ALS update, the fit
against a dense residual, and exact recovery of a rank-R tensor.
"""
import itertools

import numpy as np
import pytest

import oracle
import synth
from conftest import golden_path


# --------------------------------------------------------------------------
# helpers (independent of the oracle)
# --------------------------------------------------------------------------

def dense(dims, idx, vals):
    X = np.zeros(dims)
    for k in range(len(vals)):
        X[tuple(int(c[k]) for c in idx)] += float(vals[k])
    return X


def krp(mats):
    """Khatri-Rao product, first operand major: rows (i0, i1, ...) with i0
    slowest, (A (.) B)[i*J + j, r] = A[i, r] B[j, r]."""
    out = mats[0]
    for m in mats[1:]:
        out = (out[:, None, :] * m[None, :, :]).reshape(-1, m.shape[1])
    return out


def paper_unfold_and_krp(X, Y, d):
    """Eq. 1 operand order generalised cyclically: mode d pairs the unfolding
    whose columns sweep modes d+1, d+2, ..., d-1 (first one slowest) with
    Y_{d+1} (.) Y_{d+2} (.) ... (.) Y_{d-1}.  For N = 3 this is exactly
    X_(0)(B (.) C), X_(1)(C (.) A), X_(2)(A (.) B)."""
    N = X.ndim
    order = [(d + s) % N for s in range(N)]
    Xd = np.transpose(X, order).reshape(X.shape[d], -1)
    return Xd, krp([Y[w] for w in order[1:]])


def kolda_unfold_and_krp(X, Y, d):
    """Kolda & Bader: X_(d) columns with the lowest remaining mode fastest,
    paired with Y_{N-1} (.) ... (.) Y_{d+1} (.) Y_{d-1} (.) ... (.) Y_0."""
    N = X.ndim
    Xd = np.moveaxis(X, d, 0).reshape(X.shape[d], -1, order="F")
    rest = [w for w in range(N - 1, -1, -1) if w != d]
    return Xd, krp([Y[w] for w in rest])


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def read_golden(name):
    rows = {}
    for line in open(golden_path(name)):
        line = line.split("#")[0].split()
        if not line:
            continue
        rows.setdefault(line[0], []).append([float(t) for t in line[1:]])
    return {k: np.asarray(v) for k, v in rows.items()}


# --------------------------------------------------------------------------
# MTTKRP
# --------------------------------------------------------------------------

def test_handworked_example():
    g = read_golden("handworked_2x2x2.txt")
    nz = g["nnz"]
    idx = [nz[:, w].astype(np.int32) for w in range(3)]
    vals = nz[:, 3]
    Y = [g["A"], g["B"], g["C"]]
    for d in range(3):
        M = oracle.mttkrp((2, 2, 2), idx, vals, Y, d)
        np.testing.assert_array_equal(M, g[f"M{d}"])
        perm = oracle.mode_permutation(idx, d)
        np.testing.assert_array_equal(perm, g[f"PERM{d}"][0].astype(np.int64))


@pytest.mark.parametrize("dims", [(3, 4, 5), (2, 3, 4, 3), (2, 3, 2, 2, 3),
                                  (5, 1, 4)])
@pytest.mark.parametrize("rank", [1, 3, 8])
def test_dense_bruteforce_both_unfoldings(dims, rank):
    g = np.random.default_rng(17 + len(dims) + rank)
    nnz = max(1, int(0.4 * np.prod(dims)))
    idx = [g.integers(0, n, nnz).astype(np.int32) for n in dims]  # duplicates
    vals = g.random(nnz)
    Y = [g.standard_normal((n, rank)) for n in dims]
    X = dense(dims, idx, vals)
    for d in range(len(dims)):
        M = oracle.mttkrp(dims, idx, vals, Y, d)
        Xd, K = paper_unfold_and_krp(X, Y, d)
        assert rel(M, Xd @ K) < 1e-13
        Xd, K = kolda_unfold_and_krp(X, Y, d)
        assert rel(M, Xd @ K) < 1e-13


def test_paper_eq1_three_modes_explicit():
    """Eq. 1 written out for N = 3 with named operands A, B, C."""
    g = np.random.default_rng(3)
    I, J, K, R = 4, 3, 5, 2
    idx = [g.integers(0, n, 30).astype(np.int32) for n in (I, J, K)]
    vals = g.random(30)
    A, B, C = (g.standard_normal((n, R)) for n in (I, J, K))
    X = dense((I, J, K), idx, vals)
    X0 = X.reshape(I, J * K)                       # columns (j, k), j slowest
    X1 = X.transpose(1, 2, 0).reshape(J, K * I)    # columns (k, i)
    X2 = X.transpose(2, 0, 1).reshape(K, I * J)    # columns (i, j)
    BC = np.stack([np.kron(B[:, r], C[:, r]) for r in range(R)], 1)
    CA = np.stack([np.kron(C[:, r], A[:, r]) for r in range(R)], 1)
    AB = np.stack([np.kron(A[:, r], B[:, r]) for r in range(R)], 1)
    assert rel(oracle.mttkrp((I, J, K), idx, vals, [A, B, C], 0), X0 @ BC) < 1e-13
    assert rel(oracle.mttkrp((I, J, K), idx, vals, [A, B, C], 1), X1 @ CA) < 1e-13
    assert rel(oracle.mttkrp((I, J, K), idx, vals, [A, B, C], 2), X2 @ AB) < 1e-13


@pytest.mark.parametrize("N", [3, 4])
def test_rank1_closed_form(N):
    """X = x_0 o x_1 o ... on supp(x_0) x supp(x_1) x ...:
    M_d(i, r) = x_d(i) * prod_{w != d} (x_w . Y_w(:, r))."""
    g = np.random.default_rng(11 + N)
    dims = (7, 6, 5, 4)[:N]
    R = 3
    xs = []
    for n in dims:
        x = np.zeros(n)
        sup = g.choice(n, size=max(1, n // 2), replace=False)
        x[sup] = g.standard_normal(sup.size)
        xs.append(x)
    supports = [np.nonzero(x)[0] for x in xs]
    cells = list(itertools.product(*supports))
    idx = [np.asarray([c[w] for c in cells], dtype=np.int32) for w in range(N)]
    vals = np.asarray([np.prod([xs[w][c[w]] for w in range(N)]) for c in cells])
    Y = [g.standard_normal((n, R)) for n in dims]
    for d in range(N):
        expect = np.outer(xs[d], np.prod([xs[w] @ Y[w] for w in range(N)
                                          if w != d], axis=0))
        assert rel(oracle.mttkrp(dims, idx, vals, Y, d), expect) < 1e-13


def test_invariants_linearity_duplicates_order_inner():
    g = np.random.default_rng(5)
    dims, R, nnz = (9, 7, 8), 4, 120
    idx = [g.integers(0, n, nnz).astype(np.int32) for n in dims]
    v1, v2 = g.random(nnz), g.random(nnz)
    Y = [g.standard_normal((n, R)) for n in dims]
    Y2 = [g.standard_normal((n, R)) for n in dims]
    for d in range(3):
        # linear in the values
        a = oracle.mttkrp(dims, idx, 2.0 * v1 - 3.0 * v2, Y, d)
        b = 2.0 * oracle.mttkrp(dims, idx, v1, Y, d) - 3.0 * oracle.mttkrp(dims, idx, v2, Y, d)
        assert rel(a, b) < 1e-13
        # linear in each input factor
        w = (d + 1) % 3
        Ya = list(Y); Ya[w] = Y[w] + 0.5 * Y2[w]
        Yb = list(Y); Yb[w] = Y2[w]
        a = oracle.mttkrp(dims, idx, v1, Ya, d)
        b = oracle.mttkrp(dims, idx, v1, Y, d) + 0.5 * oracle.mttkrp(dims, idx, v1, Yb, d)
        assert rel(a, b) < 1e-13
        # the output factor is never read
        Yc = list(Y); Yc[d] = np.full_like(Y[d], np.nan)
        assert rel(oracle.mttkrp(dims, idx, v1, Yc, d), oracle.mttkrp(dims, idx, v1, Y, d)) == 0
        # input order does not matter
        p = g.permutation(nnz)
        a = oracle.mttkrp(dims, [c[p] for c in idx], v1[p], Y, d)
        assert rel(a, oracle.mttkrp(dims, idx, v1, Y, d)) < 1e-13
    # duplicates equal one summed entry
    idx_d = [np.concatenate([c, c[:10]]) for c in idx]
    v_d = np.concatenate([v1, v2[:10]])
    v_s = v1.copy(); v_s[:10] += v2[:10]
    for d in range(3):
        assert rel(oracle.mttkrp(dims, idx_d, v_d, Y, d),
                   oracle.mttkrp(dims, idx, v_s, Y, d)) < 1e-13
    # <M_d, Y_d> column by column is the same for every mode (= <X, rank-1 terms>)
    cols = [np.sum(oracle.mttkrp(dims, idx, v1, Y, d) * Y[d], axis=0) for d in range(3)]
    direct = np.zeros(R)
    for k in range(nnz):
        direct += v1[k] * np.prod([Y[w][idx[w][k]] for w in range(3)], axis=0)
    for c in cols:
        assert rel(c, direct) < 1e-12


def test_openmp_variant_is_the_same_sum():
    """The all-core baseline evaluates the same definition: one thread gives
    oracle_mttkrp's result bitwise (same terms in the same order), several
    threads regroup the FP64 sum only; bad indices are rejected."""
    try:
        oracle.build_omp()
    except oracle.OracleError as e:
        pytest.skip(str(e))
    dims, idx, vals = synth.coo_distinct((300, 200, 100, 7), 20000, (1.1, 1.1, None, None), seed=9)
    Y = synth.factors(dims, 8, seed=9)
    for d in range(4):
        ref = oracle.mttkrp(dims, idx, vals, Y, d)
        one, t1 = oracle.mttkrp_omp(dims, idx, vals, Y, d, threads=1)
        assert t1 == 1 and np.array_equal(one, ref)
        many, t = oracle.mttkrp_omp(dims, idx, vals, Y, d, threads=4)
        assert t == 4 and rel(many, ref) < 1e-13
    bad = [c.copy() for c in idx]
    bad[2][5] = dims[2]
    with pytest.raises(oracle.OracleError):
        oracle.mttkrp_omp(dims, bad, vals, Y, 0, threads=3)


def test_rows_subset_matches_full():
    dims, idx, vals = synth.coo_random((30, 20, 10), 500, seed=4, duplicates=True)
    Y = synth.factors(dims, 5, seed=4)
    rows = np.array([0, 3, 29, 17], dtype=np.int32)
    for d, r in [(0, rows), (1, rows[:3] % 20), (2, np.array([9, 0]))]:
        full = oracle.mttkrp(dims, idx, vals, Y, d)
        part = oracle.mttkrp_rows(dims, idx, vals, Y, d, r)
        np.testing.assert_array_equal(part, full[r])


def test_index_out_of_range_rejected():
    idx = [np.array([0, 5], np.int32), np.array([0, 0], np.int32)]
    with pytest.raises(oracle.OracleError):
        oracle.mttkrp((4, 2), idx, np.ones(2), [np.ones((4, 1)), np.ones((2, 1))], 0)


# --------------------------------------------------------------------------
# copy order (permutation) and partitions
# --------------------------------------------------------------------------

@pytest.mark.parametrize("dims", [(4, 3, 5), (3, 3, 3, 2), (2, 2, 2, 2, 2)])
def test_permutation_against_python_sorted(dims):
    g = np.random.default_rng(len(dims))
    nnz = 60
    idx = [g.integers(0, n, nnz).astype(np.int32) for n in dims]  # with ties
    N = len(dims)
    for d in range(N):
        keyed = sorted(range(nnz), key=lambda k: (int(idx[d][k]),) + tuple(
            int(idx[w][k]) for w in range(N) if w != d) + (k,))
        np.testing.assert_array_equal(oracle.mode_permutation(idx, d), keyed)


def test_permutation_properties_medium():
    dims, idx, vals = synth.coo_distinct((300, 200, 100), 20000, (1.2, 1.2, None), seed=9)
    for d in range(3):
        p = oracle.mode_permutation(idx, d)
        assert np.array_equal(np.sort(p), np.arange(p.size))
        keys = [idx[d][p]] + [idx[w][p] for w in range(3) if w != d]
        lex = np.lexsort(keys[::-1])           # numpy's own stable ordering
        assert np.array_equal(lex, np.arange(p.size))


@pytest.mark.parametrize("nnz,kappa", [(0, 4), (10, 3), (7, 7), (5, 9), (1000003, 152)])
def test_partition_equal(nnz, kappa):
    off = oracle.partition_equal(nnz, kappa)
    assert off[0] == 0 and off[-1] == nnz and off.size == kappa + 1
    sizes = np.diff(off)
    assert np.all(sizes >= 0) and sizes.max() - sizes.min() <= 1
    assert all(off[z] == (z * nnz) // kappa for z in range(kappa + 1))


@pytest.mark.parametrize("parts,row_cost", [(1, 4), (7, 4), (64, 4), (13, 0), (300, 9)])
def test_partition_balanced_defining_property(parts, row_cost):
    """Each boundary is the first position whose prefix cost reaches its share
    (checked directly from per-nonzero costs, not through the oracle's prefix
    sweep), boundaries are monotone, and every unit's cost is within one
    nonzero's cost of the ideal share."""
    dims, idx, vals = synth.coo_distinct((400, 90, 30), 5000, (1.2, 1.0, None), seed=parts)
    for d in range(3):
        off = oracle.partition_balanced(idx, d, parts, row_cost)
        rows = idx[d][oracle.mode_permutation(idx, d)]
        cost = np.ones(rows.size, dtype=np.int64)
        cost[0] += row_cost
        cost[1:] += row_cost * (rows[1:] != rows[:-1])
        C = np.concatenate([[0], np.cumsum(cost)])
        total = C[-1]
        assert off[0] == 0 and off[-1] == rows.size and np.all(np.diff(off) >= 0)
        for j in range(parts + 1):
            k = off[j]
            assert C[k] * parts >= j * total
            assert k == 0 or C[k - 1] * parts < j * total
        unit_cost = C[off[1:]] - C[off[:-1]]
        assert unit_cost.max() <= total / parts + 1 + row_cost


def test_partition_balanced_zero_row_cost_is_equal_split():
    dims, idx, vals = synth.coo_random((50, 40, 30), 997, seed=3, duplicates=True)
    for parts in (1, 5, 64, 2000):
        off = oracle.partition_balanced(idx, 1, parts, row_cost=0)
        assert np.array_equal(off, [-((-j * 997) // parts) for j in range(parts + 1)])


@pytest.mark.parametrize("sizes,units", [
    ([0], 4), ([10], 3), ([7, 0, 12], 7), ([5, 9, 1], 9), ([128, 129, 3000], 16),
    ([1_000_003, 17, 0, 44_444], 128)])
def test_units_from_partitions(sizes, units):
    """Work units of a partition vector, pinned without the oracle's formula:
    item k of a partition of L items belongs to unit ceil((k+1)*U/L) - 1 (the
    largest w with w*L/U <= k), counted item by item; hence every unit starts
    at its partition's offset plus the items of the earlier units, the sizes
    inside a partition differ by at most one and add up to the partition
    size."""
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    got = oracle.units_from_partitions(off, units)
    assert got.size == (off.size - 1) * units + 1 and got[-1] == off[-1]
    for z, L in enumerate(sizes):
        cnt = [0] * units
        for k in range(min(L, 3000)):
            cnt[-((-(k + 1) * units) // L) - 1] += 1
        mine = got[z * units:(z + 1) * units + 1]
        sz = np.diff(mine)
        assert mine[0] == off[z] and mine[-1] == off[z + 1]
        assert sz.sum() == L and np.all(sz >= 0)
        assert sz.max() - sz.min() <= 1
        if L <= 3000:
            assert list(sz) == cnt
        else:  # sampled items (both ends and random ones) lie in their unit
            ks = np.unique(np.concatenate([np.arange(50), L - 1 - np.arange(50),
                                           np.random.default_rng(L).integers(0, L, 2000)]))
            for k in ks:
                w = -((-(int(k) + 1) * units) // L) - 1
                assert mine[w] <= off[z] + k < mine[w + 1]


@pytest.mark.parametrize("kappa", [1, 3, 5, 40])
def test_partition_scheme1_bruteforce(kappa):
    dims, idx, vals = synth.coo_random((23, 7, 6), 200, seed=kappa, duplicates=True)
    d = 0
    perm, off, row_part = oracle.partition_scheme1(dims, idx, d, kappa)
    deg = {}
    for c in idx[d]:
        deg[int(c)] = deg.get(int(c), 0) + 1
    ordered = sorted(deg, key=lambda i: (-deg[i], i))
    expect_part = {i: t % kappa for t, i in enumerate(ordered)}
    for i in range(dims[d]):
        assert row_part[i] == expect_part.get(i, -1)
    keyed = sorted(range(200), key=lambda k: (expect_part[int(idx[d][k])], int(idx[0][k]),
                                              int(idx[1][k]), int(idx[2][k]), k))
    np.testing.assert_array_equal(perm, keyed)
    # each row sits in exactly one partition; offsets delimit the partitions
    for z in range(kappa):
        rows = idx[d][perm[off[z]:off[z + 1]]]
        assert all(expect_part[int(r)] == z for r in rows)
    assert off[-1] == 200


def test_adaptive_rule():
    assert oracle.adaptive_policy(152, 152) == 1
    assert oracle.adaptive_policy(151, 152) == 2
    assert oracle.adaptive_policy(24, 152) == 2


# --------------------------------------------------------------------------
# storage rounding
# --------------------------------------------------------------------------

def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    g = np.random.default_rng(0)
    x = np.concatenate([g.standard_normal(5000).astype(np.float32),
                        np.array([1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -2.5, 0.0,
                                  3.0e38, 1e-40, np.inf, -np.inf], np.float32)])
    ours = oracle.store_round(x.astype(np.float64), "bf16")
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(ours, ref)
    assert np.isnan(oracle.store_round(np.nan, "bf16"))
    y = g.standard_normal(100)
    np.testing.assert_array_equal(oracle.store_round(y, "fp32"),
                                  y.astype(np.float32).astype(np.float64))


# --------------------------------------------------------------------------
# CP-ALS
# --------------------------------------------------------------------------

def test_als_update_satisfies_normal_equations():
    """After the update, Z = Y_d diag(lambda) solves Z V = M_d with
    V = Hadamard of the other Grams (checked with numpy, not the oracle)."""
    dims, idx, vals = synth.coo_random((12, 10, 9), 300, seed=2, duplicates=True)
    R = 4
    Y = [f.astype(np.float64) for f in synth.factors(dims, R, seed=2)]
    for d in range(3):
        M = oracle.mttkrp(dims, idx, vals, Y, d)
        newY, lam = oracle.als_update(dims, Y, d, M, prec="fp64")
        V = np.ones((R, R))
        for w in range(3):
            if w != d:
                V *= Y[w].T @ Y[w]
        Z = newY[d] * lam[None, :]
        assert rel(Z @ V, M) < 1e-10
        assert np.allclose(np.linalg.norm(newY[d], axis=0), 1.0)
        assert np.allclose(lam, np.linalg.norm(np.linalg.solve(V, M.T).T, axis=0))
        for w in range(3):
            if w != d:
                np.testing.assert_array_equal(newY[w], Y[w])


def test_als_update_rejects_singular():
    dims = (4, 3, 3)
    Y = [np.ones((n, 2)) for n in dims]          # rank-deficient Grams
    M = np.ones((4, 2))
    with pytest.raises(oracle.OracleError):
        oracle.als_update(dims, Y, 0, M)


def test_fit_matches_dense_residual():
    dims, idx, vals = synth.coo_random((6, 5, 4), 50, seed=8, duplicates=True)
    R = 3
    Y0 = [f.astype(np.float64) for f in synth.factors(dims, R, seed=8)]
    for sweeps in (1, 2, 4):
        fac, lam, fit = oracle.cpd_als(dims, idx, vals, Y0, sweeps, prec="fp64")
        X = dense(dims, idx, vals)
        Xh = np.einsum("r,ir,jr,kr->ijk", lam, *fac)
        expect = 1.0 - np.linalg.norm(X - Xh) / np.linalg.norm(X)
        assert abs(fit[-1] - expect) < 1e-10


def test_fit_non_decreasing_fp64():
    dims, idx, vals = synth.coo_random((10, 9, 8), 200, seed=21, duplicates=True)
    Y0 = [f.astype(np.float64) for f in synth.factors(dims, 4, seed=21)]
    _, _, fit = oracle.cpd_als(dims, idx, vals, Y0, 12, prec="fp64")
    assert np.all(np.diff(fit) > -1e-12)


@pytest.mark.parametrize("R,block,dims", [(3, 3, (10, 11, 12)), (4, 3, (12, 13, 14)),
                                          (5, 3, (16, 17, 18))])
def test_exact_recovery_rank_r(R, block, dims):
    """ALS is a local method: from some random starts it stalls at a
    stationary point.  As is usual for CPD, several random starts are run and
    the best must recover the exactly rank-R tensor."""
    dims, idx, vals, true = synth.rank_r_blocks(dims, R, block, seed=4)
    best = 0.0
    for seed in range(4):
        Y0 = [f.astype(np.float64) for f in synth.factors(dims, R, seed=seed)]
        _, _, fit = oracle.cpd_als(dims, idx, vals, Y0, 60, prec="fp64")
        best = max(best, fit[-1])
    assert best > 0.9999


def test_rank1_recovered_in_two_sweeps():
    dims, idx, vals, true = synth.rank_r_blocks((5, 6, 7), 1, 4, seed=1)
    Y0 = [np.abs(f.astype(np.float64)) + 0.1 for f in synth.factors(dims, 1, seed=1)]
    _, _, fit = oracle.cpd_als(dims, idx, vals, Y0, 2, prec="fp64")
    # the fit formula subtracts squared norms, so FP64 resolves it to ~1e-8
    assert fit[-1] > 1 - 1e-7


def test_norm2_sums_duplicates():
    idx = [np.array([0, 0, 1], np.int32), np.array([1, 1, 0], np.int32)]
    assert oracle.norm2(idx, np.array([1.0, 2.0, 4.0])) == 9.0 + 16.0
