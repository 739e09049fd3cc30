"""The seeded generators: shapes, ranges, distinctness and determinism."""
import numpy as np
import pytest

import synth


def test_plain_preset():
    dims, idx, vals, R, Y = synth.preset("plain")
    assert dims == (64, 48, 32) and R == 16 and vals.size == 4096
    lin = (idx[0].astype(np.int64) * 48 + idx[1]) * 32 + idx[2]
    assert np.unique(lin).size == 4096
    assert all(c.dtype == np.int32 and c.min() >= 0 and c.max() < n
               for c, n in zip(idx, dims))
    assert vals.dtype == np.float32 and 0 <= vals.min() and vals.max() < 1
    assert [y.shape for y in Y] == [(64, 16), (48, 16), (32, 16)]
    d2, i2, v2, _, _ = synth.preset("plain")
    assert all(np.array_equal(a, b) for a, b in zip(idx, i2))


def test_zipf_distinct_small():
    dims, idx, vals = synth.coo_distinct((1000, 500, 200), 20000, (1.2, 1.2, 1.2), seed=2)
    lin = (idx[0].astype(np.int64) * 500 + idx[1]) * 200 + idx[2]
    assert np.unique(lin).size == 20000
    # heavy head: index 0 is the most frequent in every mode
    for c in idx:
        assert np.argmax(np.bincount(c)) == 0


def test_torch_generator_cpu():
    torch = pytest.importorskip("torch")
    dims, idx, vals = synth.coo_distinct_torch((300, 200, 24), 5000, (1.0, 1.0, None),
                                               seed=3, values="lognormal")
    lin = (idx[0].long() * 200 + idx[1].long()) * 24 + idx[2].long()
    assert torch.unique(lin).numel() == 5000
    assert vals.dtype == torch.float32 and bool((vals > 0).all())
    d2, i2, v2 = synth.coo_distinct_torch((300, 200, 24), 5000, (1.0, 1.0, None),
                                          seed=3, values="lognormal")
    assert all(torch.equal(a, b) for a, b in zip(idx, i2)) and torch.equal(vals, v2)


def test_rank_r_blocks_exact():
    dims, idx, vals, true = synth.rank_r_blocks((8, 9, 10), 2, 3, seed=0)
    X = np.zeros(dims)
    for k in range(vals.size):
        X[idx[0][k], idx[1][k], idx[2][k]] += vals[k]
    Xh = np.einsum("ir,jr,kr->ijk", *true)
    assert np.allclose(X, Xh)
