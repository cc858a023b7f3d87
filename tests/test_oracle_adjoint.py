"""Pins for the oracle's TTM-chain adjoint: the dot-product identity against the
(independently pinned) forward, and FP64 central finite differences."""
import numpy as np
import pytest

from oracle import tucker_oracle as O


def _rand_coo(rng, L, nnz):
    flat = rng.choice(int(np.prod(L)), size=nnz, replace=False)
    idx = np.array(np.unravel_index(flat, L, order="F"), dtype=np.int64)
    return idx, rng.random(nnz)


@pytest.mark.parametrize("L,K", [((6, 5, 4), (2, 3, 2)), ((4, 3, 5, 3), (2, 2, 3, 2))])
def test_dot_product_identity_values(L, K):
    """<ttm_chain(v), W> = <v, dval(W)>: the value-adjoint is the transpose of eq. (1)."""
    rng = np.random.default_rng(1)
    idx, _ = _rand_coo(rng, L, 40)
    F = [rng.standard_normal((l, k)) for l, k in zip(L, K)]
    v = rng.standard_normal(40)
    for n in range(len(L)):
        W = rng.standard_normal((L[n], O.khat(K, n)))
        lhs = np.sum(O.ttm_chain(L, idx, v, F, n) * W)
        dval, _ = O.ttm_chain_adjoint(L, idx, v, F, n, W)
        assert abs(lhs - v @ dval) < 1e-12 * max(1.0, abs(lhs))


def test_factor_adjoint_central_differences():
    """dF_m of <ttm_chain(F), W> against central differences, h = 1e-6 max(1,|x|)."""
    rng = np.random.default_rng(2)
    L, K = (7, 6, 5), (3, 2, 4)
    idx, vals = _rand_coo(rng, L, 50)
    F = [rng.standard_normal((l, k)) for l, k in zip(L, K)]
    for n in range(3):
        W = rng.standard_normal((L[n], O.khat(K, n)))
        _, dF = O.ttm_chain_adjoint(L, idx, vals, F, n, W)
        for m in range(3):
            if m == n:
                assert dF[m] is None
                continue
            for (i, k) in [(int(idx[m][0]), 0), (int(idx[m][7]), K[m] - 1), (int(idx[m][13]), 1)]:
                x = F[m][i, k]
                h = 1e-6 * max(1.0, abs(x))
                Fp = [f.copy() for f in F]
                Fm = [f.copy() for f in F]
                Fp[m][i, k] = x + h
                Fm[m][i, k] = x - h
                fd = (np.sum(O.ttm_chain(L, idx, vals, Fp, n) * W) - np.sum(O.ttm_chain(L, idx, vals, Fm, n) * W)) / (2 * h)
                assert abs(fd - dF[m][i, k]) < 1e-7 * max(1.0, abs(fd))


def test_factor_adjoint_zero_on_untouched_rows():
    rng = np.random.default_rng(3)
    L, K = (6, 9, 5), (2, 2, 2)
    idx, vals = _rand_coo(rng, L, 12)
    F = [rng.standard_normal((l, k)) for l, k in zip(L, K)]
    W = rng.standard_normal((L[0], O.khat(K, 0)))
    _, dF = O.ttm_chain_adjoint(L, idx, vals, F, 0, W)
    untouched = np.setdiff1d(np.arange(L[1]), idx[1])
    assert len(untouched) > 0
    assert not np.any(dF[1][untouched])
