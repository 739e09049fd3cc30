"""Error bounds of the CP-ALS row passes on the tensor cores (Sec. II-A5's
update, computed with exact operand splitting: integer digits in BF16,
exact FP32 accumulation, double-float combination).

The library's kernels run on caller data (spm_selftest_tc_rowpass):
W = V^-1 by the FP64 Cholesky, Z = M W, lambda = column norms of Z,
Y = Z / lambda and G = Y^T Y.  Each result is checked against FP64 numpy with
the bound the arithmetic guarantees:
  * Z within 2^-34 max_s|M(i,s)| sum_s|W(s,c)| (digit truncation of M and W,
    dropped levels), plus the FP64 conditioning of V^-1 and the final FP32
    rounding of Z;
  * lambda equal to the 2-norms of the returned Z to double-float accuracy;
  * Y bit-exact: the FP32 product of Z and the FP32 reciprocal of lambda;
  * G within 2^-29 (2^g_r |Y_s|_1 + 2^g_s |Y_r|_1) of the FP64 Gram of the
    stored Y, 2^g_r at most 4.1 times the column's max |Y| (column scale).
Inputs are ill-conditioned on purpose (cond(V) up to 1e6) and the rows of M
span six decades of magnitude (per-row digit scaling), with some zero rows.
"""
import numpy as np
import pytest
import torch

import paper_2503_18198_gb300 as spm

pytestmark = pytest.mark.gpu


def make_case(R, I, cond, seed):
    rng = np.random.default_rng(seed)
    M = rng.standard_normal((I, R)) * 10.0 ** rng.uniform(-3, 3, size=(I, 1))
    M[rng.choice(I, size=I // 50, replace=False)] = 0.0  # rows without nonzeros
    M = M.astype(np.float32)
    Q, _ = np.linalg.qr(rng.standard_normal((R, R)))
    V = (Q * np.logspace(0, np.log10(cond), R)) @ Q.T
    V = 0.5 * (V + V.T)
    return M, V


@pytest.mark.parametrize("R", [16, 32, 64])
@pytest.mark.parametrize("cond", [1e1, 1e4, 1e6])
def test_rowpass_within_the_splitting_bounds(R, cond):
    I = 3000 + 37  # 24 tiles of 128 rows, the last one ragged
    M, V = make_case(R, I, cond, seed=R * 10 + int(np.log10(cond)))
    Z, Y, G, lam = spm.spm_selftest_tc_rowpass(torch.from_numpy(M).cuda(),
                                               torch.from_numpy(V).cuda())
    Z = Z.cpu().numpy().astype(np.float64)
    Y = Y.cpu().numpy()
    G = G.cpu().numpy()
    lam = lam.cpu().numpy()

    W = np.linalg.inv(V)
    M64 = M.astype(np.float64)
    Zref = M64 @ W
    scale = np.abs(M64).max(axis=1, keepdims=True) * np.abs(W).sum(axis=0, keepdims=True)
    bound = (2.0 ** -34 + cond * R * 2.0 ** -50) * scale + 2.0 ** -23 * np.abs(Zref) + 1e-300
    err = np.abs(Z - Zref)
    assert np.all(err <= bound), float((err / bound).max())
    assert np.all(Z[np.abs(M64).sum(axis=1) == 0] == 0.0)  # zero rows stay exactly zero

    ref_lam = np.sqrt((Z * Z).sum(axis=0))
    assert np.allclose(lam, ref_lam, rtol=1e-11, atol=0.0)

    inv = (1.0 / lam).astype(np.float32)
    Yref = Z.astype(np.float32) * inv[None, :]
    assert np.array_equal(Y.view(np.uint32), Yref.view(np.uint32))

    if R <= 32:
        Y64 = Y.astype(np.float64)
        Gref = Y64.T @ Y64
        amax = np.abs(Y64).max(axis=0)
        l1 = np.abs(Y64).sum(axis=0)
        gb = 2.0 ** -29 * 4.1 * (amax[:, None] * l1[None, :] + amax[None, :] * l1[:, None])
        gb = gb + 1e-12 * np.abs(Gref).max()
        assert np.all(np.abs(G - Gref) <= gb), float((np.abs(G - Gref) / gb).max())
        assert np.array_equal(G, G.T)  # written from the lower triangle
        assert np.allclose(np.diag(G), 1.0, rtol=1e-6)  # unit columns after normalisation


def test_rowpass_rejects_a_system_that_is_not_positive_definite():
    R, I = 32, 256
    M = torch.randn(I, R, device="cuda")
    V = -torch.eye(R, dtype=torch.float64, device="cuda")
    with pytest.raises(spm.SpmError) as e:
        spm.spm_selftest_tc_rowpass(M, V)
    assert e.value.status == 5  # SPM_ERR_NUMERIC


def test_rowpass_rejects_other_ranks():
    M = torch.randn(64, 8, device="cuda")
    V = torch.eye(8, dtype=torch.float64, device="cuda")
    with pytest.raises(spm.SpmError):
        spm.spm_selftest_tc_rowpass(M, V)
