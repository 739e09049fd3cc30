"""Element-wise parity bound of an FP32-accumulated MTTKRP against the oracle.

An output element M_d(i, r) is a sum of terms t_k = val_k * prod_w Y_w(c_w, r)
over the nonzeros of row i.  Any floating-point evaluation of that sum (each
term rounded a few times, the terms added in some tree of depth D) is within
about (D + N) * 2^-24 * sum_k |t_k| of the exact value, so the natural
per-element bound is relative to the sum of the magnitudes of the terms --
the MTTKRP of |val| and |Y|, which the oracle computes by the same
definition on those inputs.  A wrong row, a dropped or doubled term, a
missing empty-row clear or a partial row lost at a boundary shows up in its
own element, however small the row is next to the heavy (Zipf-head) rows
that dominate a Frobenius norm.

TOL_ELEM = 1e-5 is the worst case of a chain of ~160 FP32 additions, each
rounding by a full half-ulp in the same direction.  The kernels' chains (one
slot's share of a work unit -- a few hundred terms at the 50M-nonzero size --
then shuffle, block and partition trees) round in both directions, so their
error grows like a random walk, about 2^-24 * sqrt(depth) of the magnitudes,
far inside the bound.  Elements whose terms are all zero (empty rows) must
be exactly zero.
"""
import numpy as np

import oracle

TOL_ELEM = 1e-5


def abs_inputs(vals, factors):
    return (np.abs(np.asarray(vals, np.float64)),
            [np.abs(np.asarray(f, np.float64)) for f in factors])


def assert_elementwise(got, ref, absref, tol=TOL_ELEM, what=""):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    absref = np.asarray(absref, np.float64)
    assert got.shape == ref.shape == absref.shape
    err = np.abs(got - ref)
    bad = err > tol * absref
    if bad.any():
        i = np.argwhere(bad)[0]
        raise AssertionError(
            f"{what}: {int(bad.sum())} elements outside tol * sum|terms|; first at {tuple(i)}: "
            f"got {got[tuple(i)]!r} ref {ref[tuple(i)]!r} sum|terms| {absref[tuple(i)]!r}")


def check_mode_elementwise(got, dims, idx, vals, factors, d, tol=TOL_ELEM, what=""):
    """Whole output of mode d against the oracle, element by element."""
    ref = oracle.mttkrp(dims, idx, vals, factors, d)
    av, af = abs_inputs(vals, factors)
    absref = oracle.mttkrp(dims, idx, av, af, d)
    assert_elementwise(got, ref, absref, tol, what or f"mode {d}")
    return ref


def check_rows_elementwise(got_rows, dims, idx, vals, factors, d, rows, tol=TOL_ELEM, what=""):
    """Sampled output rows `rows` of mode d, element by element."""
    ref = oracle.mttkrp_rows(dims, idx, vals, factors, d, rows)
    av, af = abs_inputs(vals, factors)
    absref = oracle.mttkrp_rows(dims, idx, av, af, d, rows)
    assert_elementwise(got_rows, ref, absref, tol, what or f"mode {d} rows")
    return ref
